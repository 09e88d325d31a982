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
#include "level1.h"
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"
#include "solver.h"

using namespace ddtm;
typedef std::complex<double> zc;

namespace ddtm {

void validate_params(ddtm_ctx* c, const ddtm_params& p) {
  if (p.n_levels != 2 && p.n_levels != 3) throw Error(DDTM_ERR_ARG, "n_levels must be 2 or 3");
  if (p.n_levels == 3) {
    if (p.nv[1] < 1 || p.nv[1] > 32) throw Error(DDTM_ERR_ARG, "nv[1] must be in 1..32");
    for (int m = 0; m < 4; m++)
      if (p.block[1][m] < 1 || c->g.NB[m] % p.block[1][m] || (c->g.NB[m] / p.block[1][m]) % 2)
        throw Error(DDTM_ERR_ARG, "block[1] must divide the level-1 lattice into an even number of blocks per "
                                  "direction");
    if (p.kcycle_restart < 1 || p.kcycle_restart > 64 || p.kcycle_max_restarts < 0 || !(p.kcycle_tol > 0))
      throw Error(DDTM_ERR_ARG, "invalid K-cycle parameters");
  }
  for (int m = 0; m < 4; m++)
    if (p.block[0][m] != c->g.b[m]) throw Error(DDTM_ERR_ARG, "block[0] is fixed at ddtm_create");
  if (p.nv[0] < 1 || p.nv[0] > 64) throw Error(DDTM_ERR_ARG, "nv[0] must be in 1..64");
  if (p.n_setup < 1 || p.post_smooth < 0 || p.nmr < 1) throw Error(DDTM_ERR_ARG, "invalid smoother/setup counts");
  if (p.coarse_restart < 1 || p.coarse_restart > 250 || p.coarse_max_restarts < 0 || p.outer_restart < 1 ||
      p.outer_restart > 250 || p.outer_max_iters < 1)
    throw Error(DDTM_ERR_ARG, "invalid Krylov parameters");
  if (!(p.outer_tol > 0) || !(p.coarse_tol > 0) || !(p.delta > 0) || !(p.restart_tol > 0))
    throw Error(DDTM_ERR_ARG, "invalid tolerances");
  if (p.smoother_prec != DDTM_PREC_F64 && p.smoother_prec != DDTM_PREC_F32 && p.smoother_prec != DDTM_PREC_F16)
    throw Error(DDTM_ERR_ARG, "smoother_prec must be F64, F32 or F16");
  if (p.coarse_prec != DDTM_PREC_F32 && p.coarse_prec != DDTM_PREC_F16)
    throw Error(DDTM_ERR_ARG, "coarse_prec must be F32 or F16");
  if (p.coarse_prec == DDTM_PREC_F16 && p.nv[0] > 32)
    throw Error(DDTM_ERR_ARG, "coarse_prec F16 (tensor-core coarse stencil) needs nv[0] <= 32");
}

void invalidate_setup(ddtm_ctx* c) {
  c->setup_done = false;
  c->have_P = false;
  c->c1.built = false;
  c->c1.inv_valid = false;
  c->c2.built = false;
  c->c2.inv_valid = false;
}

// the level whose operator the even-odd GMRES of Sec. 2.5 inverts (with the shifted twist)
static CoarseLevel& coarsest(ddtm_ctx* c) { return c->p.n_levels == 3 ? c->c2 : c->c1; }

// right-hand sides per batch of the level-0 transfers of the C ABI
static const int ABI_BATCH = 12;

void sap_run(ddtm_ctx* c, int prec, void* x, float* xn, const void* b, const float* bn, double mu, int ncycles, int nmr,
             bool from_zero, int R) {
  ensure_fine_prec(c, prec);
  ensure_site_inverse(c, prec, mu);
  const FineGeom& g = c->g;
  int half = g.Nb / 2;
  const int* red = g.colour_blocks.as<int>();
  const int* black = red + half;
  if (ncycles <= 0) {
    if (from_zero) {
      CK(cudaMemsetAsync(x, 0, (size_t)R * g.V * 12 * store2_bytes(prec), c->stream));
      if (xn) CK(cudaMemsetAsync(xn, 0, (size_t)R * g.V * sizeof(float), c->stream));
    }
    return;
  }
  for (int cyc = 0; cyc < ncycles; cyc++) {
    launch_sap_half(g, prec, x, xn, b, bn, c->links[prec].p, c->clover[prec].p, c->sinv[prec].p, red, black, half,
                    from_zero && cyc == 0, nmr, mu, R, c->stream);
    launch_sap_half(g, prec, x, xn, b, bn, c->links[prec].p, c->clover[prec].p, c->sinv[prec].p, black, red, half, 0,
                    nmr, mu, R, c->stream);
  }
}

// ---- hierarchy -----------------------------------------------------------------------
static size_t fine_field_bytes(const FineGeom& g, int prec) { return (size_t)g.V * 12 * store2_bytes(prec); }

// coarse batches are padded with zero columns to a multiple of 4 right-hand
// sides (register blocking of the coarse kernels) that the interleaved vector
// kernels take: lcm(R, 32) <= 256, i.e. R / gcd(R, 32) <= 8 (so R <= 256)
static bool interleave_ok(int R) {
  int a = R, b = 32;
  while (b) { int t = a % b; a = b; b = t; }
  return R / a <= 8;
}
int coarse_batch(int R) {
  if (R == 1) return 1;
  int r = (R + 3) / 4 * 4;
  while (r <= kMaxBatch && !interleave_ok(r)) r += 4;
  if (r > kMaxBatch) throw Error(DDTM_ERR_ARG, "internal: coarse batch of " + std::to_string(R) + " right-hand sides");
  return r;
}

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
  // with three levels, level 1 (the K-cycle's operator, SIMT) stays FP32; only the coarsest level
  // runs on the tensor cores
  L.prec = c->p.n_levels == 3 ? PREC_F32 : c->p.coarse_prec;
  L.Dc.ensure((size_t)L.Nc * 9 * L.n * L.n * 8);
  launch_galerkin(g, c->faces, PREC_F32, L.Dc.p, c->P0.as<float2>(), c->links[PREC_F32].p, c->clover[PREC_F32].p, nv,
                  L.prec == PREC_F16, c->stream);
  if (L.prec == PREC_F16) build_coarse_images(L, c->stream);
  L.inv_valid = false;
  L.built = true;
  c->have_P = true;
}

// P_1 from the level-1 test vectors, then D_2 = P_1^+ D_1 P_1 (three levels)
void build_hierarchy1(ddtm_ctx* c) {
  CoarseLevel& L1 = c->c1;
  Level1Agg& a = c->a1;
  if (!a.geom) build_level1_aggregates(L1, c->p.block[1], a);
  launch_l1_build_P(a, L1, c->stream);
  CoarseLevel& L2 = c->c2;
  if (!c->c2_geom) {
    build_coarse_geometry_lat(a.NB, L2);
    c->c2_geom = true;
  }
  L2.nv = a.nv;
  L2.n = 2 * a.nv;
  L2.prec = c->p.coarse_prec;
  launch_l1_galerkin(a, L1, L2, c->scratch, c->stream);
  if (L2.prec == PREC_F16) build_coarse_images(L2, c->stream);
  L2.inv_valid = false;
  L2.built = true;
}

void require_hierarchy(ddtm_ctx* c) {
  require_gauge(c);
  if (!c->have_P || !c->c1.built || (c->p.n_levels == 3 && !c->c2.built))
    throw Error(DDTM_ERR_STATE, "no aggregation / coarse operator (call ddtm_setup)");
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

// ---- batched GMRES on FP32 vectors --------------------------------------------------------
// A(out, in) applies the operator to a batch of R interleaved vectors.
// The input is a batch of vectors of type tag in_type (1 FP32, 2 FP16; see blas.h).
typedef std::function<void(cplx<float>*, const void*, int)> OpF32;

// Runs body() (kernel launches on c->stream and on the Blas stream *bst) as a
// CUDA graph keyed by key: the first time a key is met in an allocation
// generation the launches run directly (they may allocate); the second time
// they are captured on the context's private capture stream, instantiated and
// replayed; afterwards every call is one graph launch on c->stream.  The key
// must name everything the launches' arguments depend on besides device
// buffers (their addresses are fixed within a generation).
static void run_as_graph(ddtm_ctx* c, const std::string& key, cudaStream_t* bst, const std::function<void()>& body) {
  if (!c->use_graphs || timer_on() || tc_forced_wait_ns()) {  // a forced tensor-core timeout is never captured
    body();
    return;
  }
  const long gen = alloc_generation();
  if (gen != c->graphs_gen) {  // buffers moved: every cached graph is stale
    for (auto& kv : c->graphs)
      if (kv.second.first) cudaGraphExecDestroy(kv.second.first);
    c->graphs.clear();
    c->graphs_gen = gen;
  }
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    body();
    if (alloc_generation() == gen) c->graphs.emplace(key, std::make_pair((cudaGraphExec_t) nullptr, 0));
    return;
  }
  if (it->second.first) {
    CK(cudaGraphLaunch(it->second.first, c->stream));
    add_kernel_launches(it->second.second);
    return;
  }
  if (!c->capture_stream) CK(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
  // the capture stream starts after everything issued so far on c->stream
  cudaEvent_t ev[2];
  c->events("graph_capture", ev);
  CK(cudaEventRecord(ev[0], c->stream));
  CK(cudaStreamWaitEvent(c->capture_stream, ev[0], 0));
  const cudaStream_t saved = c->stream, saved_b = *bst;
  cudaGraph_t graph = nullptr;
  const long before = kernel_launches();
  c->stream = *bst = c->capture_stream;
  CK(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
  try {
    body();
  } catch (...) {
    cudaStreamEndCapture(c->capture_stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    c->stream = saved;
    *bst = saved_b;
    throw;
  }
  const cudaError_t ec = cudaStreamEndCapture(c->capture_stream, &graph);
  c->stream = saved;
  *bst = saved_b;
  CK(ec);
  const long nk = kernel_launches() - before;  // counted once now, for the replay below
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(ei);
  it->second = std::make_pair(exec, (int)nk);
  CK(cudaGraphLaunch(exec, c->stream));
}

// Lockstep GMRES(m) with restarts for R systems A x_r = b_r (complex FP32
// vectors of L entries each, interleaved; FP64 inner products).  Every
// iteration orthogonalises all R Krylov vectors with one multi-dot and one
// fused multi-axpy + norm (classical Gram-Schmidt; a second pass when tol is
// below 1e-3).  The Hessenberg matrices, Givens rotations and least-squares
// updates stay on the device, so an iteration issues kernels only; the host
// reads the residual estimates one iteration behind (asynchronous copy and an
// event) and stops when every system is below tol (systems with b_r = 0 count
// as solved with x_r = 0).  An iteration already issued when the stop is seen
// is discarded: the solution uses exactly the columns up to the converged one.
// x is overwritten (zero start).  Returns the iteration count; relres[r] the
// final estimates.  half_basis: the Krylov basis is stored in FP16 (the
// residual, the new vector before normalisation and x stay FP32); every
// product with it is formed in FP32, so the Arnoldi relation holds to FP16
// rounding of the basis, far below the loose tolerances of the coarsest solve.
// With a preconditioner M (flexible GMRES, the K-cycle solver of intermediate
// levels, Sec. 2.5): z_j = M v_j is kept (FP32) and w = A z_j; the update is
// x += sum_j y_j z_j.
static int gmres_b(ddtm_ctx* c, const OpF32& A, cplx<float>* x, const cplx<float>* b, size_t L, int R, int m, int max_restarts,
                   double tol, double* relres, const char* tag, bool half_basis, const std::string& op_key,
                   const OpF32* M = nullptr) {
  Blas B(c->stream, &c->scratch, &c->ring);
  std::string t(tag);
  const size_t N = L * R;
  if (M) half_basis = false;
  const int vt = half_basis ? 2 : 1;
  const size_t vb = half_basis ? sizeof(__half2) : sizeof(float2);
  char* V = (char*)c->scratch.get(t + (half_basis ? "_Vh" : "_V"), (size_t)(m + 1) * N * vb);
  auto Vj = [&](int j) { return (void*)(V + (size_t)j * N * vb); };
  float2* Z = M ? (float2*)c->scratch.get(t + "_Z", (size_t)m * N * sizeof(float2)) : nullptr;
  auto Zj = [&](int j) { return (cplx<float>*)(Z + (size_t)j * N); };
  cplx<float>* w = (cplx<float>*)c->scratch.get(t + "_w", N * sizeof(float2));
  // device bookkeeping, one block of scratch
  size_t nH = (size_t)R * (m + 1) * m, ncs = (size_t)R * m, ng = (size_t)R * (m + 1), nh = (size_t)(m + 1) * R;
  size_t tot2 = nH + 2 * ncs + ng + 3 * nh + 3 * (size_t)R;
  double2* st2 = (double2*)c->scratch.get(t + "_state", tot2 * sizeof(double2) + 2 * (size_t)R * sizeof(double));
  ArnoldiDev ad;
  ad.H = st2;
  ad.cs = ad.H + nH;
  ad.sn = ad.cs + ncs;
  ad.g = ad.sn + ncs;
  double2* h = ad.g + ng;
  double2* h2 = h + nh;
  double2* y = h2 + nh;
  double2* nr2 = y + nh;
  ad.scale = nr2 + R;  // (one more block of R stays reserved after it)
  ad.bn = (double*)(st2 + tot2);
  ad.est = ad.bn + R;
  ad.m = m;
  ad.R = R;
  // pinned mirrors of the estimates, double-buffered by iteration parity
  double* est_h = (double*)c->scratch_host(t + "_est", 2 * (size_t)R * sizeof(double));
  cudaEvent_t ev[2];
  c->events(t, ev);

  CK(cudaMemsetAsync(x, 0, N * sizeof(float2), c->stream));
  auto vs = [&](const void* p) { return VSet{(void*)p, 1, L, R, true}; };
  auto vsb = [&](const void* p) { return VSet{(void*)p, vt, L, R, true}; };
  std::vector<double> bn(R);
  B.norms2(vs(b), bn.data());
  for (int r = 0; r < R; r++) bn[r] = sqrt(bn[r]);
  CK(cudaMemcpyAsync(ad.bn, bn.data(), R * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const bool reorth = tol < 1e-3;
  std::vector<double2> one(R, make_double2(1, 0)), mone(R, make_double2(-1, 0));
  std::vector<double> est(R, 0.0);
  auto all_done = [&](const double* e) {
    for (int r = 0; r < R; r++) {
      if (!std::isfinite(e[r])) throw Error(DDTM_ERR_NAN, "non-finite residual in GMRES (" + t + ")");
      if (bn[r] > 0 && !(e[r] <= tol)) return false;
    }
    return true;
  };
  auto fetch_est = [&](int slot) {
    CK(cudaMemcpyAsync(est_h + (size_t)slot * R, ad.est, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(ev[slot], c->stream));
  };
  int iters = 0;
  bool done = false;
  for (int cyc = 0; cyc <= max_restarts && !done; cyc++) {
    // residual in w (FP32), then V_0 = w / ||w||
    if (cyc == 0) {
      CK(cudaMemcpyAsync(w, b, N * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      A(w, x, 1);
      B.axpby(one.data(), vs(b), mone.data(), vs(w));
    }
    B.dots_dev(vs(w), 0, 1, vs(w), nr2);
    launch_arnoldi_start(ad, nr2, c->stream);
    fetch_est(0);
    CK(cudaEventSynchronize(ev[0]));
    for (int r = 0; r < R; r++) est[r] = est_h[r];
    if (all_done(est.data())) break;
    B.scale_dev(ad.scale, vs(w), vsb(Vj(0)));
    int k = 0;
    for (int j = 0; j < m; j++) {
      auto iteration = [&]() {
        if (M) {
          (*M)(Zj(j), Vj(j), vt);
          A(w, Zj(j), 1);
        } else {
          A(w, Vj(j), vt);
        }
        B.dots_dev(vsb(V), N, j + 1, vs(w), h);
        B.maxpy_dev(vs(w), vsb(V), N, j + 1, h, -1.0, reorth ? nullptr : nr2);
        if (reorth) {
          B.dots_dev(vsb(V), N, j + 1, vs(w), h2);
          B.maxpy_dev(vs(w), vsb(V), N, j + 1, h2, -1.0, nr2);
        }
        launch_arnoldi_step(ad, j, h, reorth ? h2 : nullptr, nr2, c->stream, tol >= 1e-3);
        CK(cudaMemcpyAsync(est_h + (size_t)(j & 1) * R, ad.est, R * sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        if (j < m - 1) B.scale_dev(ad.scale, vs(w), vsb(Vj(j + 1)));  // V_{j+1} = w / ||w||
      };
      if (op_key.empty() || M) {
        iteration();
      } else {
        char kb[160];
        snprintf(kb, sizeof(kb), "%s|j%d|R%d|m%d|L%zu|%d%d|est%p|", t.c_str(), j, R, m, L, (int)reorth,
                 (int)half_basis, (void*)est_h);
        run_as_graph(c, std::string(kb) + op_key, &B.st, iteration);
      }
      CK(cudaEventRecord(ev[j & 1], c->stream));
      iters++;
      k = j + 1;
      if (j >= 1) {  // estimates of the previous iteration
        CK(cudaEventSynchronize(ev[(j - 1) & 1]));
        const double* e = est_h + (size_t)((j - 1) & 1) * R;
        if (all_done(e)) {
          for (int r = 0; r < R; r++) est[r] = e[r];
          k = j;  // iteration j is discarded
          iters--;
          done = true;
          break;
        }
      }
    }
    if (!done) {
      CK(cudaEventSynchronize(ev[(k - 1) & 1]));
      const double* e = est_h + (size_t)((k - 1) & 1) * R;
      for (int r = 0; r < R; r++) est[r] = e[r];
      done = all_done(est.data());
    }
    launch_arnoldi_solve(ad, k, y, c->stream);
    if (M) B.maxpy_dev(vs(x), vs(Z), N, k, y, +1.0, nullptr);
    else B.maxpy_dev(vs(x), vsb(V), N, k, y, +1.0, nullptr);
  }
  for (int r = 0; r < R; r++) relres[r] = est[r];
  return iters;
}

// ---- coarsest level: even-odd GMRES (Sec. 2.5) ------------------------------------------
// D_c(mu_c) phi = eta for a batch of Rc interleaved coarse vectors:
// rhat = eta_o - D_oe D_ee^-1 eta_e;  GMRES on D_hat = D_oo - D_oe D_ee^-1 D_eo;
// phi_e = D_ee^-1 (eta_e - D_eo phi_o).  Returns the iteration count; relres
// receives the per-rhs estimates of the reduced system.
int coarse_eo_solve(ddtm_ctx* c, cplx<float>* x_full, const cplx<float>* b_full, int Rc, double mu_c, int restart,
                    int max_restarts, double tol, double* relres) {
  CoarseLevel& L = coarsest(c);
  if (!L.inv_valid || L.inv_mu != mu_c) launch_self_inverse(L, mu_c, c->stream);
  size_t ne = L.h_even.size(), no = L.h_odd.size(), n = L.n;
  size_t bytes_e = ne * n * Rc * 8, bytes_o = no * n * Rc * 8;
  cplx<float>* be = (cplx<float>*)c->scratch.get("ceo_be", bytes_e);
  cplx<float>* bo = (cplx<float>*)c->scratch.get("ceo_bo", bytes_o);
  cplx<float>* te = (cplx<float>*)c->scratch.get("ceo_te", bytes_e);
  cplx<float>* xo = (cplx<float>*)c->scratch.get("ceo_xo", bytes_o);
  cplx<float>* tA = (cplx<float>*)c->scratch.get("ceo_tA", bytes_e);
  launch_parity_copy(L, 0, be, (cplx<float>*)b_full, Rc, 0, c->stream);
  launch_parity_copy(L, 1, bo, (cplx<float>*)b_full, Rc, 0, c->stream);
  launch_coarse_even(L, te, be, nullptr, Rc, 1.f, 0.f, c->stream);                 // te = D_ee^-1 eta_e
  launch_coarse_apply_odd(L, bo, nullptr, te, Rc, mu_c, 2, -1.f, 1.f, c->stream);   // rhat = eta_o - D_oe te
  OpF32 Dhat;
  if (L.prec == PREC_F16) {
    // tensor cores: FP16 images of the operand vectors, FP32 accumulation;
    // only the input and the output of D_hat are FP32 vectors
    const size_t img_o = tc_vector_image_bytes(L, (int)no, Rc), img_e = tc_vector_image_bytes(L, (int)ne, Rc);
    char* vt = (char*)c->scratch.get("ceo_vt", img_o);
    char* tt = (char*)c->scratch.get("ceo_tt", img_e);
    const size_t ab = tc_geom(L.n, 1).a_bytes;
    Dhat = [&, vt, tt, ab](cplx<float>* out, const void* in, int in_type) {
      launch_vector_image(L, vt, in, in_type, (int)no, Rc, c->stream);
      TcPass h;  // tt = -D_ee^-1 D_eo in, from the products D_ee^-1(e) A_d(e) (one pass, no intermediate)
      h.name = "coarse_tc_hop_even";
      h.hops = true;
      h.A_hop = L.Dhopt.p;
      h.hop_by_slot = true;
      h.X_hop = vt;
      h.tab = L.nbr_eo.as<int>();
      h.osite = L.even.as<int>();
      h.nout = (int)ne;
      h.sres = -1.f;
      h.yt = tt;
      launch_coarse_tc(L, h, Rc, c->stream);
      TcPass o;  // out = (D_oo + i mu_c Gamma5_c) in + D_oe tt
      o.name = "coarse_tc_odd";
      o.self = o.hops = true;
      o.A_self = L.Dct.p;
      o.a_self_stride = 9 * ab;
      o.self_by_site = true;
      o.A_hop = L.Dct.p;
      o.X_self = vt;
      o.X_hop = tt;
      o.tab = L.nbr_oe.as<int>();
      o.osite = L.odd.as<int>();
      o.nout = (int)no;
      o.y = out;
      o.xs = in;
      o.xs_type = in_type;
      o.mu_c = (float)mu_c;
      launch_coarse_tc(L, o, Rc, c->stream);
    };
  } else {
    Dhat = [&](cplx<float>* out, const void* in_v, int in_type) {
      if (in_type != 1) throw Error(DDTM_ERR_ARG, "internal: FP32 coarse stencil takes FP32 vectors");
      const cplx<float>* in = (const cplx<float>*)in_v;
      launch_coarse_even(L, tA, nullptr, in, Rc, 0.f, -1.f, c->stream);               // tA = -D_ee^-1 D_eo in
      launch_coarse_apply_odd(L, out, in, tA, Rc, mu_c, 3, 1.f, 0.f, c->stream);      // out = D_oo in + D_oe tA
    };
  }
  // FP16 Krylov basis with the tensor-core stencil (which reads FP16 operands anyway)
  char ok[96];  // what the operator's launch arguments depend on besides buffers
  snprintf(ok, sizeof(ok), "eo|mu%.17g|p%d|lev%p", mu_c, L.prec, (const void*)&L);
  int it = gmres_b(c, Dhat, xo, bo, no * n, Rc, restart, max_restarts, tol, relres, "cgm", L.prec == PREC_F16,
                   std::string(ok));
  launch_coarse_even(L, te, be, xo, Rc, 1.f, -1.f, c->stream);  // phi_e = D_ee^-1 (eta_e - D_eo phi_o)
  launch_parity_copy(L, 0, te, x_full, Rc, 1, c->stream);
  launch_parity_copy(L, 1, xo, x_full, Rc, 1, c->stream);
  c->coarse_iters += (long)it * Rc;
  return it;
}

// ---- level 1 of three (Sec. 2.2 K-cycle on the intermediate level) ------------------------
// SAP on D_1(mu) for Rc interleaved level-1 vectors (Rc a multiple of 4): ncycles red-black
// cycles, from x = 0 if from_zero, else from x
static void sap_l1(ddtm_ctx* c, cplx<float>* x, const cplx<float>* b, double mu, int ncycles, int nmr, bool from_zero,
                   int Rc) {
  CoarseLevel& L1 = c->c1;
  if (!c->a1.geom) build_level1_aggregates(L1, c->p.block[1], c->a1);  // the SAP blocks are the aggregates
  if (from_zero) CK(cudaMemsetAsync(x, 0, (size_t)L1.Nc * L1.n * Rc * 8, c->stream));
  for (int cyc = 0; cyc < ncycles; cyc++) {
    launch_l1_sap_half(c->a1, L1, (float2*)x, (const float2*)b, 0, mu, nmr, Rc, c->stream);
    launch_l1_sap_half(c->a1, L1, (float2*)x, (const float2*)b, 1, mu, nmr, Rc, c->stream);
  }
}

// One application of the level-1 preconditioner: z = P_1 D_2(delta mu)^-1 R_1 v (even-odd GMRES on
// the coarsest level), then post_smooth SAP cycles on D_1(mu) z = v started from that z.
static void precondition_l1(ddtm_ctx* c, cplx<float>* z, const cplx<float>* v, double mu, int Rc) {
  CoarseLevel& L2 = c->c2;
  const size_t n2 = (size_t)L2.Nc * L2.n * Rc;
  cplx<float>* c2 = (cplx<float>*)c->scratch.get("l1_c2", n2 * 8);
  cplx<float>* e2 = (cplx<float>*)c->scratch.get("l1_e2", n2 * 8);
  launch_l1_restrict(c->a1, c->c1, (float2*)c2, (const float2*)v, Rc, Rc, c->stream);
  std::vector<double> rr(Rc);
  coarse_eo_solve(c, e2, c2, Rc, c->p.delta * mu, c->p.coarse_restart, c->p.coarse_max_restarts, c->p.coarse_tol,
                  rr.data());
  launch_l1_prolong(c->a1, c->c1, (float2*)z, (const float2*)e2, Rc, Rc, 0, c->stream);
  sap_l1(c, z, v, mu, c->p.post_smooth, c->p.nmr, false, Rc);
}

// x ~ D_1(mu)^-1 b: flexible GMRES(kcycle_restart) with kcycle_max_restarts restarts to
// kcycle_tol, preconditioned by precondition_l1 (Table 1: FGMRES(5), 2 restarts, 1e-1)
static void kcycle_l1(ddtm_ctx* c, cplx<float>* x, const cplx<float>* b, double mu, int Rc) {
  CoarseLevel& L1 = c->c1;
  OpF32 A = [&](cplx<float>* out, const void* in, int in_type) {
    if (in_type != 1) throw Error(DDTM_ERR_ARG, "internal: level-1 operator takes FP32 vectors");
    launch_coarse_apply_full(L1, out, (const cplx<float>*)in, Rc, mu, 3, 1.f, 0.f, c->stream);
  };
  OpF32 M = [&](cplx<float>* out, const void* in, int in_type) {
    if (in_type != 1) throw Error(DDTM_ERR_ARG, "internal: level-1 preconditioner takes FP32 vectors");
    precondition_l1(c, out, (const cplx<float>*)in, mu, Rc);
  };
  std::vector<double> rr(Rc);
  gmres_b(c, A, x, b, (size_t)L1.Nc * L1.n, Rc, c->p.kcycle_restart, c->p.kcycle_max_restarts, c->p.kcycle_tol,
          rr.data(), "kc1", false, std::string(), &M);
}

// ---- K-cycle preconditioner (Sec. 2.2): z = P D_c^-1 R v, then post-smoothing ----------
// R fine fields of precision prec at stride 12 V (FP16 scales at stride V).
void mg_precondition(ddtm_ctx* c, int prec, void* z, float* zn, const void* v, const float* vn, double mu, int R) {
  const FineGeom& g = c->g;
  CoarseLevel& L = c->c1;
  // the level-1 SAP of three levels works on chunks of 4 right-hand sides
  const int Rc = c->p.n_levels == 3 && coarse_batch(R) < 4 ? 4 : coarse_batch(R);
  size_t nc = (size_t)L.Nc * L.n * Rc;
  cplx<float>* cv = (cplx<float>*)c->scratch.get("mg_c", nc * 8);
  cplx<float>* ev = (cplx<float>*)c->scratch.get("mg_e", nc * 8);
  if (Rc != R) CK(cudaMemsetAsync(cv, 0, nc * 8, c->stream));
  int pprec;
  const void* P = P_for(c, prec, &pprec);
  launch_restrict(g, prec, cv, v, vn, P, pprec, L.nv, R, Rc, c->stream);
  if (c->p.n_levels == 3) {
    kcycle_l1(c, ev, cv, mu, Rc);  // level 1 keeps the twist mu; the coarsest level uses delta mu
  } else {
    std::vector<double> rr(Rc);
    coarse_eo_solve(c, ev, cv, Rc, c->p.delta * mu, c->p.coarse_restart, c->p.coarse_max_restarts, c->p.coarse_tol,
                    rr.data());
  }
  launch_prolong(g, prec, z, zn, ev, P, pprec, L.nv, R, Rc, 0, c->stream);
  sap_run(c, prec, z, zn, v, vn, mu, c->p.post_smooth, c->p.nmr, false, R);
}

// ---- outer mixed-precision flexible GMRES (Sec. 2.5, Table 1) ---------------------------
// R systems in lockstep, as iterative refinement around an FP32 flexible GMRES
// cycle: every cycle starts from the true FP64 residual r = b - D x (FP64
// operator), runs flexible GMRES on r with the Arnoldi basis, the operator
// applications w = D z and the Gram-Schmidt products in FP32 (inner products
// summed in FP64), and ends with the FP64 update x += sum_j y_j Z_j.  A cycle
// stops when every system's estimate fell below restart_tol times its
// starting residual (Table 1's mixed-precision restarting criterion) or
// below the final target, or at the restart length.  Z_j = M v_j is stored in
// the smoother precision: the flexible method uses exactly the stored Z_j for
// both w = D Z_j and the update.  Hessenberg matrices and Givens rotations stay
// on the device; the host reads the estimates one iteration behind.
// With an FP64 smoother the cycle itself is FP64 (basis, w = D z, Gram-Schmidt)
// and runs to the final target: the plain FP64 method, kept as the reference
// for the mixed-precision solver (the coarse correction stays FP32).
struct OuterResult {
  int iters = 0, restarts = 0;
  std::vector<double> relres;
  bool converged = false;
};

OuterResult outer_fgmres(ddtm_ctx* c, double* x, const double* b, double mu, int R) {
  const FineGeom& g = c->g;
  const ddtm_params& p = c->p;
  Blas B(c->stream, &c->scratch, &c->ring);
  const int sp = p.smoother_prec, m = p.outer_restart;
  const size_t n = (size_t)g.V * 12;  // complex entries of one fine field
  const size_t fb = fine_field_bytes(g, sp);
  // cycle precision: FP32 (mixed precision) or, with an FP64 smoother, FP64 throughout
  const bool c64 = sp == PREC_F64;
  const int cp = c64 ? PREC_F64 : PREC_F32, vt = c64 ? 0 : 1;
  const size_t cb = n * (c64 ? 16 : 8);  // bytes of one cycle-precision field
  ensure_fine_prec(c, cp);
  char* V = (char*)c->scratch.get(c64 ? "out_V64" : "out_V", (size_t)(m + 1) * R * cb);
  char* Z = (char*)c->scratch.get("out_Z", (size_t)m * R * fb);
  float* Zn = (float*)c->scratch.get("out_Zn", (size_t)m * R * g.V * sizeof(float));
  char* w = (char*)c->scratch.get(c64 ? "out_w64" : "out_w", (size_t)R * cb);
  char* t32 = (char*)c->scratch.get(c64 ? "out_t64c" : "out_t32", (size_t)R * cb);
  double* r64 = (double*)c->scratch.get("out_r64", (size_t)R * n * 16);
  char* vsb = (char*)c->scratch.get("out_vs", (size_t)R * fb);
  float* vsn = (float*)c->scratch.get("out_vsn", (size_t)R * g.V * sizeof(float));
  auto Zj = [&](int j) { return (void*)(Z + (size_t)j * R * fb); };
  auto Zjn = [&](int j) { return sp == PREC_F16 ? Zn + (size_t)j * R * g.V : (float*)nullptr; };
  auto Vj = [&](int j) { return (void*)(V + (size_t)j * R * cb); };
  auto s64 = [&](const double* p0) { return VSet{(void*)p0, 0, n, R, false}; };
  auto sc_ = [&](const void* p0) { return VSet{(void*)p0, vt, n, R, false}; };
  auto D64 = [&](double* out, const double* in) {
    for (int r = 0; r < R; r++)
      launch_dslash(g, PREC_F64, out + 2 * (size_t)r * n, nullptr, in + 2 * (size_t)r * n, nullptr, c->links[0].p,
                    c->clover[0].p, mu, c->stream);
  };
  auto Dcyc = [&](void* out, const void* in) {  // all R right-hand sides in one launch where possible
    launch_dslash_multi(g, cp, out, nullptr, in, nullptr, c->links[cp].p, c->clover[cp].p, mu, R, c->stream);
  };
  // device bookkeeping
  size_t nH = (size_t)R * (m + 1) * m, ncs = (size_t)R * m, ng = (size_t)R * (m + 1), nh = (size_t)(m + 1) * R;
  size_t tot2 = nH + 2 * ncs + ng + 3 * nh + 2 * (size_t)R;
  double2* st2 = (double2*)c->scratch.get("out_state", tot2 * sizeof(double2) + 2 * (size_t)R * sizeof(double));
  ArnoldiDev ad;
  ad.H = st2;
  ad.cs = ad.H + nH;
  ad.sn = ad.cs + ncs;
  ad.g = ad.sn + ncs;
  double2* h = ad.g + ng;
  double2* h2 = h + nh;
  double2* y = h2 + nh;
  double2* nr2 = y + nh;
  ad.scale = nr2 + R;
  ad.bn = (double*)(st2 + tot2);
  ad.est = ad.bn + R;
  ad.m = m;
  ad.R = R;
  double* est_h = (double*)c->scratch_host("out_est", 2 * (size_t)R * sizeof(double));
  cudaEvent_t ev[2];
  c->events("out", ev);

  OuterResult res;
  res.relres.assign(R, 1.0);
  std::vector<double> bn(R), beta(R), thr(R);
  B.norms2(s64(b), bn.data());
  for (int r = 0; r < R; r++) bn[r] = sqrt(bn[r]);
  CK(cudaMemsetAsync(x, 0, (size_t)R * n * 16, c->stream));
  std::vector<double2> one(R, make_double2(1, 0)), mone(R, make_double2(-1, 0)), zero(R, make_double2(0, 0)), sc(R);
  auto fetch_est = [&](int slot) {
    CK(cudaMemcpyAsync(est_h + (size_t)slot * R, ad.est, R * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(ev[slot], c->stream));
  };
  auto cycle_done = [&](const double* e) {
    for (int r = 0; r < R; r++) {
      if (!std::isfinite(e[r])) throw Error(DDTM_ERR_NAN, "non-finite outer residual estimate");
      if (!(e[r] <= thr[r])) return false;
    }
    return true;
  };
  bool first = true;
  while (true) {
    // true residual in FP64
    CK(cudaMemcpyAsync(r64, b, (size_t)R * n * 16, cudaMemcpyDeviceToDevice, c->stream));
    if (!first) {
      double* t64 = (double*)c->scratch.get("out_t64", (size_t)R * n * 16);
      D64(t64, x);
      B.axpby(mone.data(), s64(t64), one.data(), s64(r64));
      res.restarts++;
    }
    first = false;
    B.norms2(s64(r64), beta.data());
    bool done = true;
    for (int r = 0; r < R; r++) {
      beta[r] = sqrt(beta[r]);
      res.relres[r] = bn[r] > 0 ? beta[r] / bn[r] : 0.0;
      if (!std::isfinite(res.relres[r])) throw Error(DDTM_ERR_NAN, "non-finite outer residual");
      done = done && res.relres[r] <= p.outer_tol;
      sc[r] = make_double2(beta[r] > 0 ? 1.0 / beta[r] : 0.0, 0);
      // stop the cycle at restart_tol relative to its start, or at the final target
      // (an FP64 cycle needs no restarts for precision: it runs to the target)
      const double target = 0.5 * p.outer_tol * bn[r] / beta[r];
      thr[r] = beta[r] > 0 ? (c64 ? target : std::max(p.restart_tol, target)) : 1.0;
    }
    if (done) {
      res.converged = true;
      break;
    }
    if (res.iters >= p.outer_max_iters) break;
    // V_0 = r / beta in the cycle precision; the device state starts with
    // g_0 = beta and estimates relative to beta (so y is the correction for r itself)
    B.axpby(sc.data(), s64(r64), zero.data(), sc_(Vj(0)));
    {
      double* hb = (double*)c->scratch_host("out_beta", 3 * (size_t)R * sizeof(double));
      for (int r = 0; r < R; r++) {
        hb[r] = beta[r] > 0 ? beta[r] : 1.0;       // bn: reference of the estimates
        hb[R + 2 * r] = beta[r] * beta[r];         // nr2[r].x
        hb[R + 2 * r + 1] = 0.0;                   // nr2[r].y
      }
      CK(cudaMemcpyAsync(ad.bn, hb, R * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(nr2, hb + R, 2 * (size_t)R * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      launch_arnoldi_start(ad, nr2, c->stream);
      CK(cudaStreamSynchronize(c->stream));  // the pinned block is rewritten next cycle
    }
    int k = 0;
    bool cyc_done = false;
    for (int j = 0; j < m; j++) {
      const void* vin = Vj(j);
      const float* vinn = nullptr;
      if (sp != cp) {
        for (int r = 0; r < R; r++)
          launch_field_convert(g, cp, (char*)Vj(j) + (size_t)r * cb, nullptr, sp, vsb + (size_t)r * fb,
                               sp == PREC_F16 ? vsn + (size_t)r * g.V : nullptr, c->stream);
        vin = vsb;
        vinn = sp == PREC_F16 ? vsn : nullptr;
      }
      mg_precondition(c, sp, Zj(j), Zjn(j), vin, vinn, mu, R);
      const void* zin = Zj(j);
      if (sp != cp) {
        for (int r = 0; r < R; r++)
          launch_field_convert(g, sp, (char*)Zj(j) + (size_t)r * fb, sp == PREC_F16 ? Zjn(j) + (size_t)r * g.V : nullptr,
                               cp, t32 + (size_t)r * cb, nullptr, c->stream);
        zin = t32;
      }
      Dcyc(w, zin);
      B.dots_dev(sc_(V), (size_t)R * n, j + 1, sc_(w), h);
      B.maxpy_dev(sc_(w), sc_(V), (size_t)R * n, j + 1, h, -1.0, nullptr);
      B.dots_dev(sc_(V), (size_t)R * n, j + 1, sc_(w), h2);
      B.maxpy_dev(sc_(w), sc_(V), (size_t)R * n, j + 1, h2, -1.0, nr2);
      launch_arnoldi_step(ad, j, h, h2, nr2, c->stream, false);
      fetch_est(j & 1);
      if (j < m - 1) B.scale_dev(ad.scale, sc_(w), sc_(Vj(j + 1)));
      res.iters++;
      k = j + 1;
      if (j >= 1) {
        CK(cudaEventSynchronize(ev[(j - 1) & 1]));
        if (cycle_done(est_h + (size_t)((j - 1) & 1) * R)) {
          k = j;  // iteration j is discarded
          res.iters--;
          cyc_done = true;
          break;
        }
      }
      if (res.iters >= p.outer_max_iters) break;
    }
    if (!cyc_done) CK(cudaEventSynchronize(ev[(k - 1) & 1]));
    launch_arnoldi_solve(ad, k, y, c->stream);
    // x += sum_j y_j Z_j in FP64
    double* t64 = (double*)c->scratch.get("out_t64", (size_t)R * n * 16);
    for (int j = 0; j < k; j++) {
      const double* zj = (const double*)Zj(j);
      if (sp != PREC_F64) {
        for (int r = 0; r < R; r++)
          launch_field_convert(g, sp, (char*)Zj(j) + (size_t)r * fb, sp == PREC_F16 ? Zjn(j) + (size_t)r * g.V : nullptr,
                               PREC_F64, t64 + 2 * (size_t)r * n, nullptr, c->stream);
        zj = t64;
      }
      B.maxpy_dev(s64(x), s64(zj), 0, 1, y + (size_t)j * R, +1.0, nullptr);
    }
  }
  return res;
}

// ---- adaptive setup (Sec. 2.6) -----------------------------------------------------------------
static void normalise_fields(ddtm_ctx* c, float2* tv, int nv) {
  Blas B(c->stream, &c->scratch, &c->ring);
  size_t n = (size_t)c->g.V * 12;
  VSet s{tv, 1, n, nv, false};
  std::vector<double> nn(nv);
  B.norms2(s, nn.data());
  std::vector<double2> zero(nv, make_double2(0, 0)), sc(nv);
  for (int i = 0; i < nv; i++) {
    double q = sqrt(nn[i]);
    if (!(q > 0) || !std::isfinite(q)) throw Error(DDTM_ERR_NAN, "test vector vanished or became non-finite in setup");
    sc[i] = make_double2(1.0 / q, 0);
  }
  B.axpby(zero.data(), s, sc.data(), s);
}

// Adaptive setup (Sec. 2.6).  update = false: random test vectors, one SAP pass,
// then n_setup - 1 inverse-iteration steps.  update = true (the HMC usage of
// Sec. 3.2: the setup follows a changed gauge field or twist): the existing
// test vectors are kept, P and the coarse operators are rebuilt from them and
// n_iter inverse-iteration steps follow.
void run_setup(ddtm_ctx* c, double mu, uint64_t seed, bool update = false, int n_iter = 0) {
  const FineGeom& g = c->g;
  const ddtm_params& p = c->p;
  int nv = p.nv[0];
  c->nv0 = nv;
  size_t n = (size_t)g.V * 12;
  c->tv0.ensure((size_t)nv * n * sizeof(float2));
  float2* tv = c->tv0.as<float2>();
  if (!update)
    for (int i = 0; i < nv; i++)
      launch_gaussian(tv + (size_t)i * n, n, seed * 0x100000001b3ull + (uint64_t)i * (n * 2 + 17), c->stream);
  // the setup works in the smoother precision, FP32 for an FP64 smoother
  int sp = p.smoother_prec == PREC_F64 ? PREC_F32 : p.smoother_prec;
  size_t fb = fine_field_bytes(g, sp);
  char* bs = (char*)c->scratch.get("setup_b", (size_t)nv * fb);
  float* bsn = (float*)c->scratch.get("setup_bn", (size_t)nv * g.V * 4);
  char* xs = (char*)c->scratch.get("setup_x", (size_t)nv * fb);
  float* xsn = (float*)c->scratch.get("setup_xn", (size_t)nv * g.V * 4);
  auto to_sp = [&]() {
    for (int i = 0; i < nv; i++)
      launch_field_convert(g, PREC_F32, tv + (size_t)i * n, nullptr, sp, bs + (size_t)i * fb,
                           sp == PREC_F16 ? bsn + (size_t)i * g.V : nullptr, c->stream);
  };
  auto from_sp = [&]() {
    for (int i = 0; i < nv; i++)
      launch_field_convert(g, sp, xs + (size_t)i * fb, sp == PREC_F16 ? xsn + (size_t)i * g.V : nullptr, PREC_F32,
                           tv + (size_t)i * n, nullptr, c->stream);
  };
  float* bnp = sp == PREC_F16 ? bsn : nullptr;
  float* xnp = sp == PREC_F16 ? xsn : nullptr;
  // level 1 of three: its own random vectors, batch-interleaved for the level-1 kernels
  const bool three = p.n_levels == 3;
  const int nv1 = three ? p.nv[1] : 0, R1 = three ? coarse_batch(nv1) : 0;
  float2 *tv1 = nullptr, *b1 = nullptr, *x1 = nullptr;
  size_t N1 = 0;
  if (three) {
    N1 = (size_t)g.Nb * 2 * nv;  // level-1 sites x n1
    c->a1.nv = nv1;
    c->a1.tv.ensure((size_t)nv1 * N1 * sizeof(float2));
    tv1 = c->a1.tv.as<float2>();
    if (!update)
      for (int i = 0; i < nv1; i++)
        launch_gaussian(tv1 + (size_t)i * N1, N1,
                        (seed ^ 0x5bd1e995ull) * 0x100000001b3ull + (uint64_t)i * (N1 * 2 + 29), c->stream);
    b1 = (float2*)c->scratch.get("setup_b1", N1 * R1 * sizeof(float2));
    x1 = (float2*)c->scratch.get("setup_x1", N1 * R1 * sizeof(float2));
  }
  Blas B1(c->stream, &c->scratch);
  auto normalise_l1 = [&]() {
    for (int i = 0; i < nv1; i++) {
      const double n2 = B1.norm2(tv1 + (size_t)i * N1, 1, N1);
      const double sc = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
      B1.axpby(make_double2(sc, 0), tv1 + (size_t)i * N1, 1, make_double2(0, 0), tv1 + (size_t)i * N1, 1, N1);
    }
  };
  if (update) {  // hierarchy from the kept test vectors
    build_hierarchy(c);
    if (three) build_hierarchy1(c);
  } else {
    // k = 1: the SAP smoother on every random vector, all vectors as one batch
    to_sp();
    sap_run(c, sp, xs, xnp, bs, bnp, mu, p.post_smooth, p.nmr, true, nv);
    from_sp();
    normalise_fields(c, tv, nv);
    build_hierarchy(c);
    if (three) {
      launch_l1_transpose(tv1, b1, N1, nv1, R1, 0, c->stream);
      sap_l1(c, (cplx<float>*)x1, (const cplx<float>*)b1, mu, p.post_smooth, p.nmr, true, R1);
      launch_l1_transpose(tv1, x1, N1, nv1, R1, 1, c->stream);
      normalise_l1();
      build_hierarchy1(c);
    }
  }
  // k >= 2: one multigrid iteration per test vector, all vectors as one batch (level by level)
  const int k_last = update ? n_iter + 1 : p.n_setup;
  for (int k = 2; k <= k_last; k++) {
    to_sp();
    mg_precondition(c, sp, xs, xnp, bs, bnp, mu, nv);
    from_sp();
    normalise_fields(c, tv, nv);
    build_hierarchy(c);
    if (three) {
      launch_l1_transpose(tv1, b1, N1, nv1, R1, 0, c->stream);
      precondition_l1(c, (cplx<float>*)x1, (const cplx<float>*)b1, mu, R1);
      launch_l1_transpose(tv1, x1, N1, nv1, R1, 1, c->stream);
      normalise_l1();
      build_hierarchy1(c);
    }
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

static void check_level(ddtm_ctx* c, int level, int lo, int hi_off = 0) {
  if (level < lo || level > c->p.n_levels - 1 - hi_off)
    throw Error(DDTM_ERR_ARG, "level " + std::to_string(level) + " out of range for a " +
                                  std::to_string(c->p.n_levels) + "-level hierarchy");
}
static CoarseLevel& level_op(ddtm_ctx* c, int level) { return level == 2 ? c->c2 : c->c1; }
static void check_tc_all(ddtm_ctx* c) {
  check_tc_error(c->c1);
  check_tc_error(c->c2);
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
    sap_run(ctx, prec, fx.data.p, fx.nrm.as<float>(), fb.data.p, fb.nrm.as<float>(), mu, ncycles, nmr, true, 1);
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
  sap_run(ctx, x->prec, field_ptr(x, 0), field_nrm(x, 0), field_ptr(b, 0), field_nrm(b, 0), mu, ncycles, nmr, true,
          x->nrhs);
  API_END(ctx)
}

int ddtm_setup(ddtm_ctx* ctx, double mu, uint64_t seed) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  if (!std::isfinite(mu)) throw Error(DDTM_ERR_ARG, "invalid mu");
  invalidate_setup(ctx);
  double t0 = now_s();
  run_setup(ctx, mu, seed);
  CK(cudaStreamSynchronize(ctx->stream));
  check_tc_all(ctx);
  ctx->setup_s = now_s() - t0;
  ctx->setup_done = true;
  ctx->setup_mu = mu;
  API_END(ctx)
}

int ddtm_setup_update(ddtm_ctx* ctx, double mu, int n_iter) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  if (!std::isfinite(mu) || n_iter < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  if (!ctx->tv0.p || ctx->nv0 != ctx->p.nv[0] ||
      (ctx->p.n_levels == 3 && (!ctx->a1.tv.p || ctx->a1.nv != ctx->p.nv[1])))
    throw Error(DDTM_ERR_STATE, "no test vectors of these parameters to update (call ddtm_setup first)");
  invalidate_setup(ctx);
  double t0 = now_s();
  run_setup(ctx, mu, 0, true, n_iter);
  CK(cudaStreamSynchronize(ctx->stream));
  check_tc_all(ctx);
  ctx->setup_s = now_s() - t0;
  ctx->setup_done = true;
  ctx->setup_mu = mu;
  API_END(ctx)
}

int ddtm_set_test_vectors(ddtm_ctx* ctx, int level, const double* v, int nv, int loc) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  check_loc(loc);
  check_level(ctx, level, 0, 1);
  if (!v || nv != ctx->p.nv[level]) throw Error(DDTM_ERR_ARG, "nv must equal params.nv[level]");
  if (level == 1) {
    // level-1 test vectors (canonical coarse vectors of level 1): P_1 and D_2
    if (!ctx->have_P || !ctx->c1.built) throw Error(DDTM_ERR_STATE, "set the level-0 test vectors first");
    const size_t N1 = (size_t)ctx->c1.Nc * ctx->c1.n;
    ctx->a1.nv = nv;
    ctx->a1.tv.ensure((size_t)nv * N1 * sizeof(float2));
    for (int i = 0; i < nv; i++) {
      const double* din = stage_in(ctx, "canon_cin", v + 2 * N1 * i, N1, loc);
      launch_convert_complex(din, PREC_F32, ctx->a1.tv.as<float2>() + (size_t)i * N1, N1, ctx->stream);
    }
    build_hierarchy1(ctx);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->setup_done = true;
    return DDTM_OK;
  }
  size_t nsp = (size_t)ctx->g.V * 12;
  ctx->nv0 = nv;
  ctx->tv0.ensure((size_t)nv * nsp * sizeof(float2));
  for (int i = 0; i < nv; i++) {
    const double* din = stage_in(ctx, "canon_in", v + 2 * nsp * i, nsp, loc);
    launch_spinor_from_canon(ctx->g, PREC_F32, ctx->tv0.as<float2>() + (size_t)i * nsp, nullptr, din, ctx->stream);
  }
  build_hierarchy(ctx);
  if (ctx->p.n_levels == 3 && ctx->a1.tv.p && ctx->a1.nv == ctx->p.nv[1]) build_hierarchy1(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->setup_done = ctx->p.n_levels == 2 || ctx->c2.built;
  API_END(ctx)
}

int ddtm_build_coarse(ddtm_ctx* ctx) {
  API_BEGIN(ctx)
  require_gauge(ctx);
  if (!ctx->tv0.p || ctx->nv0 <= 0) throw Error(DDTM_ERR_STATE, "no test vectors (call ddtm_setup)");
  build_hierarchy(ctx);
  if (ctx->p.n_levels == 3) {
    if (!ctx->a1.tv.p || ctx->a1.nv != ctx->p.nv[1]) throw Error(DDTM_ERR_STATE, "no level-1 test vectors");
    build_hierarchy1(ctx);
  }
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
  if (!cout || !x || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  check_level(ctx, level, 0, 1);
  require_hierarchy(ctx);
  if (level == 1) {  // level-1 vectors -> level-2 vectors, one at a time (R = 1 interleaved = canonical)
    Blas B1(ctx->stream, &ctx->scratch);
    const size_t n1 = (size_t)ctx->c1.Nc * ctx->c1.n, n2 = (size_t)ctx->c2.Nc * ctx->c2.n;
    float2* v = (float2*)ctx->scratch.get("abi_l1", n1 * 8);
    float2* c2 = (float2*)ctx->scratch.get("abi_l2", n2 * 8);
    for (int r = 0; r < nrhs; r++) {
      const double* din = stage_in(ctx, "canon_cin", x + 2 * n1 * r, n1, loc);
      double* dout = stage_out(ctx, "canon_cout", cout + 2 * n2 * r, n2, loc);
      B1.axpby(make_double2(1, 0), din, 0, make_double2(0, 0), v, 1, n1);
      launch_l1_restrict(ctx->a1, ctx->c1, c2, v, 1, 1, ctx->stream);
      B1.axpby(make_double2(1, 0), c2, 1, make_double2(0, 0), dout, 0, n2);
      unstage_out(ctx, cout + 2 * n2 * r, dout, n2, loc);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return DDTM_OK;
  }
  // batches of up to ABI_BATCH right-hand sides go through one restriction launch (the solver's
  // batched kernels, here with the FP32 P)
  const FineGeom& g = ctx->g;
  CoarseLevel& L = ctx->c1;
  size_t nsp = (size_t)g.V * 12, nc = (size_t)L.Nc * L.n;
  const int CH = nrhs < ABI_BATCH ? nrhs : ABI_BATCH;
  float2* f = (float2*)ctx->scratch.get("abi_f32", (size_t)CH * nsp * 8);
  cplx<float>* cv = (cplx<float>*)ctx->scratch.get("abi_c32", (size_t)CH * nc * 8);
  for (int r0 = 0; r0 < nrhs; r0 += CH) {
    const int R = nrhs - r0 < CH ? nrhs - r0 : CH;
    for (int rc = 0; rc < R; rc++) {
      const double* din = stage_in(ctx, "canon_in", x + 2 * nsp * (r0 + rc), nsp, loc);
      launch_spinor_from_canon(g, PREC_F32, f + (size_t)rc * nsp, nullptr, din, ctx->stream);
    }
    launch_restrict(g, PREC_F32, cv, f, nullptr, ctx->P0.p, PREC_F32, L.nv, R, R, ctx->stream);
    for (int rc = 0; rc < R; rc++) {
      double* dout = stage_out(ctx, "canon_cout", cout + 2 * nc * (r0 + rc), nc, loc);
      launch_coarse_interleave(L, cv, dout, rc, R, 1, ctx->stream);
      unstage_out(ctx, cout + 2 * nc * (r0 + rc), dout, nc, loc);
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_prolong(ddtm_ctx* ctx, int level, double* x, const double* cin, int nrhs, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!cin || !x || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  check_level(ctx, level, 0, 1);
  require_hierarchy(ctx);
  if (level == 1) {  // level-2 vectors -> level-1 vectors
    Blas B1(ctx->stream, &ctx->scratch);
    const size_t n1 = (size_t)ctx->c1.Nc * ctx->c1.n, n2 = (size_t)ctx->c2.Nc * ctx->c2.n;
    float2* v = (float2*)ctx->scratch.get("abi_l1", n1 * 8);
    float2* c2 = (float2*)ctx->scratch.get("abi_l2", n2 * 8);
    for (int r = 0; r < nrhs; r++) {
      const double* din = stage_in(ctx, "canon_cin", cin + 2 * n2 * r, n2, loc);
      double* dout = stage_out(ctx, "canon_cout", x + 2 * n1 * r, n1, loc);
      B1.axpby(make_double2(1, 0), din, 0, make_double2(0, 0), c2, 1, n2);
      launch_l1_prolong(ctx->a1, ctx->c1, v, c2, 1, 1, 0, ctx->stream);
      B1.axpby(make_double2(1, 0), v, 1, make_double2(0, 0), dout, 0, n1);
      unstage_out(ctx, x + 2 * n1 * r, dout, n1, loc);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return DDTM_OK;
  }
  const FineGeom& g = ctx->g;
  CoarseLevel& L = ctx->c1;
  size_t nsp = (size_t)g.V * 12, nc = (size_t)L.Nc * L.n;
  const int CH = nrhs < ABI_BATCH ? nrhs : ABI_BATCH;
  float2* f = (float2*)ctx->scratch.get("abi_f32", (size_t)CH * nsp * 8);
  cplx<float>* cv = (cplx<float>*)ctx->scratch.get("abi_c32", (size_t)CH * nc * 8);
  for (int r0 = 0; r0 < nrhs; r0 += CH) {
    const int R = nrhs - r0 < CH ? nrhs - r0 : CH;
    for (int rc = 0; rc < R; rc++) {
      const double* din = stage_in(ctx, "canon_cin", cin + 2 * nc * (r0 + rc), nc, loc);
      launch_coarse_interleave(L, cv, const_cast<double*>(din), rc, R, 0, ctx->stream);
    }
    launch_prolong(g, PREC_F32, f, nullptr, cv, ctx->P0.p, PREC_F32, L.nv, R, R, 0, ctx->stream);
    for (int rc = 0; rc < R; rc++) {
      double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * (r0 + rc), nsp, loc);
      launch_spinor_to_canon(g, PREC_F32, f + (size_t)rc * nsp, nullptr, dout, ctx->stream);
      unstage_out(ctx, x + 2 * nsp * (r0 + rc), dout, nsp, loc);
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  API_END(ctx)
}

int ddtm_coarse_solve_batch(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu_c, int loc, int* iters) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!x || !b || nrhs < 0 || !std::isfinite(mu_c)) throw Error(DDTM_ERR_ARG, "invalid arguments");
  require_hierarchy(ctx);
  if (iters) *iters = 0;
  if (nrhs == 0) return DDTM_OK;
  CoarseLevel& L = coarsest(ctx);
  const size_t nc = (size_t)L.Nc * L.n;
  const int Rc = coarse_batch(nrhs);  // the batch the solver's kernels take, padded with zero columns
  cplx<float>* bv = (cplx<float>*)ctx->scratch.get("abi_cb", nc * Rc * 8);
  cplx<float>* xv = (cplx<float>*)ctx->scratch.get("abi_cx", nc * Rc * 8);
  CK(cudaMemsetAsync(bv, 0, nc * Rc * 8, ctx->stream));
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_cin", b + 2 * nc * r, nc, loc);
    launch_coarse_interleave(L, bv, const_cast<double*>(din), r, Rc, 0, ctx->stream);
  }
  std::vector<double> rr(Rc, 0.0);
  const int it = coarse_eo_solve(ctx, xv, bv, Rc, mu_c, ctx->p.coarse_restart, ctx->p.coarse_max_restarts,
                                 ctx->p.coarse_tol, rr.data());
  for (int r = 0; r < nrhs; r++) {
    double* dout = stage_out(ctx, "canon_cout", x + 2 * nc * r, nc, loc);
    launch_coarse_interleave(L, xv, dout, r, Rc, 1, ctx->stream);
    unstage_out(ctx, x + 2 * nc * r, dout, nc, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  check_tc_error(L);
  if (iters) *iters = it;
  double worst = 0;
  for (int r = 0; r < nrhs; r++) worst = rr[r] > worst ? rr[r] : worst;
  if (worst > ctx->p.coarse_tol) {
    ctx->err = "coarse solve stopped at relative residual " + std::to_string(worst);
    return DDTM_ERR_NOCONV;
  }
  API_END(ctx)
}

int ddtm_apply_Dc(ddtm_ctx* ctx, int level, double* y, const double* x, int nrhs, double mu, int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!x || !y || nrhs < 0) throw Error(DDTM_ERR_ARG, "invalid arguments");
  check_level(ctx, level, 1);
  require_hierarchy(ctx);
  if (nrhs == 0) return DDTM_OK;
  CoarseLevel& L = level_op(ctx, level);
  const size_t nc = (size_t)L.Nc * L.n;
  // all right-hand sides go through one batched stencil pass
  cplx<float>* xv = (cplx<float>*)ctx->scratch.get("abi_c32", nc * nrhs * 8);
  cplx<float>* yv = (cplx<float>*)ctx->scratch.get("abi_c32b", nc * nrhs * 8);
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_cin", x + 2 * nc * r, nc, loc);
    launch_coarse_interleave(L, xv, const_cast<double*>(din), r, nrhs, 0, ctx->stream);
  }
  if (L.prec == PREC_F16) {
    char* xt = (char*)ctx->scratch.get("abi_ct", tc_vector_image_bytes(L, L.Nc, nrhs));
    launch_vector_image(L, xt, xv, 1, L.Nc, nrhs, ctx->stream);
    TcPass f;
    f.name = "coarse_tc_full";
    f.self = f.hops = true;
    f.A_self = f.A_hop = L.Dct.p;
    f.a_self_stride = 9 * (size_t)tc_geom(L.n, 1).a_bytes;
    f.X_self = f.X_hop = xt;
    f.tab = L.nbr.as<int>();
    f.nout = L.Nc;
    f.y = yv;
    f.xs = xv;
    f.mu_c = (float)mu;
    launch_coarse_tc(L, f, nrhs, ctx->stream);
  } else {
    launch_coarse_apply_full(L, yv, xv, nrhs, mu, 3, 1.f, 0.f, ctx->stream);
  }
  for (int r = 0; r < nrhs; r++) {
    double* dout = stage_out(ctx, "canon_cout", y + 2 * nc * r, nc, loc);
    launch_coarse_interleave(L, yv, dout, r, nrhs, 1, ctx->stream);
    unstage_out(ctx, y + 2 * nc * r, dout, nc, loc);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  check_tc_error(L);
  API_END(ctx)
}

int ddtm_sap_coarse(ddtm_ctx* ctx, int level, double* x, const double* b, int nrhs, double mu, int ncycles, int nmr,
                    int loc) {
  API_BEGIN(ctx)
  check_loc(loc);
  if (!x || !b || nrhs < 0 || ncycles < 0 || nmr < 1 || !std::isfinite(mu)) throw Error(DDTM_ERR_ARG, "invalid arguments");
  if (ctx->p.n_levels != 3 || level != 1) throw Error(DDTM_ERR_ARG, "SAP on a coarse level exists for level 1 of three");
  require_hierarchy(ctx);
  if (nrhs == 0) return DDTM_OK;
  CoarseLevel& L1 = ctx->c1;
  const int Rc = (nrhs + 3) / 4 * 4;
  const size_t nc = (size_t)L1.Nc * L1.n;
  cplx<float>* bv = (cplx<float>*)ctx->scratch.get("abi_sapc_b", nc * Rc * 8);
  cplx<float>* xv = (cplx<float>*)ctx->scratch.get("abi_sapc_x", nc * Rc * 8);
  CK(cudaMemsetAsync(bv, 0, nc * Rc * 8, ctx->stream));
  for (int r = 0; r < nrhs; r++) {
    const double* din = stage_in(ctx, "canon_cin", b + 2 * nc * r, nc, loc);
    launch_coarse_interleave(L1, bv, const_cast<double*>(din), r, Rc, 0, ctx->stream);
  }
  sap_l1(ctx, xv, bv, mu, ncycles, nmr, true, Rc);
  for (int r = 0; r < nrhs; r++) {
    double* dout = stage_out(ctx, "canon_cout", x + 2 * nc * r, nc, loc);
    launch_coarse_interleave(L1, xv, dout, r, Rc, 1, ctx->stream);
    unstage_out(ctx, x + 2 * nc * r, dout, nc, loc);
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
  CoarseLevel& L = coarsest(ctx);
  size_t nc = (size_t)L.Nc * L.n;
  cplx<float>* bv = (cplx<float>*)ctx->scratch.get("abi_c32", nc * 8);
  cplx<float>* xv = (cplx<float>*)ctx->scratch.get("abi_c32b", nc * 8);
  const double* din = stage_in(ctx, "canon_cin", b, nc, loc);
  double* dout = stage_out(ctx, "canon_cout", x, nc, loc);
  B.axpby(make_double2(1, 0), din, 0, make_double2(0, 0), bv, 1, nc);
  double rr;
  int it = coarse_eo_solve(ctx, xv, bv, 1, mu_c, ctx->p.coarse_restart, ctx->p.coarse_max_restarts, ctx->p.coarse_tol, &rr);
  B.axpby(make_double2(1, 0), xv, 1, make_double2(0, 0), dout, 0, nc);
  unstage_out(ctx, x, dout, nc, loc);
  CK(cudaStreamSynchronize(ctx->stream));
  check_tc_error(L);
  if (iters) *iters = it;
  if (rr > ctx->p.coarse_tol) {
    ctx->err = "coarse solve stopped at relative residual " + std::to_string(rr);
    return DDTM_ERR_NOCONV;
  }
  API_END(ctx)
}

// Right-hand sides per outer batch: all of them when the per-rhs work fields
// of the outer solver (FP64 input, output and residual, the cycle-precision
// basis of outer_restart + 1 fields, the stored preconditioned fields in the
// smoother precision, the work fields) fit in the device memory that is free
// or already held by those same buffers (they are reused or regrown), less a
// reserve of 10% of the device for everything else.
static int solve_batch(ddtm_ctx* ctx, int nrhs) {
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  const FineGeom& g = ctx->g;
  const int m = ctx->p.outer_restart, sp = ctx->p.smoother_prec;
  const size_t cyc = sp == PREC_F64 ? 16 : 8;  // bytes per complex entry of the cycle precision
  const size_t n = (size_t)g.V * 12;
  const size_t per = n * ((m + 1) * cyc + m * store2_bytes(sp) + 4 * 16 + 3 * cyc + 2 * store2_bytes(sp)) +
                     (size_t)g.V * (m + 2) * sizeof(float);
  const size_t held = ctx->scratch.held("out_") + ctx->scratch.held("solve_");
  const size_t reserve = tot / 10;
  size_t avail = fr + held > reserve ? fr + held - reserve : 0;
  const size_t cap = device_memory_limit();  // the caller's budget, if any, bounds the batch as well
  if (cap) {
    const size_t in_use = device_bytes_in_use();
    const size_t room = cap > in_use ? cap - in_use + held : held;
    if (room < avail) avail = room;
  }
  int R = per > 0 ? (int)(avail / per) : nrhs;
  if (R < 1) R = 1;
  if (R > kMaxBatch) R = kMaxBatch;  // interleaved coarse batches hold at most kMaxBatch columns
  return R < nrhs ? R : nrhs;
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
  ddtm_solve_info acc;
  memset(&acc, 0, sizeof(acc));
  ctx->coarse_iters = 0;
  bool all_conv = true;
  int batch = nrhs > 0 ? solve_batch(ctx, nrhs) : 1;
  for (int r0 = 0; r0 < nrhs; r0 += batch) {
    int R = nrhs - r0 < batch ? nrhs - r0 : batch;
    double* bf = (double*)ctx->scratch.get("solve_b", (size_t)R * nsp * 16);
    double* xf = (double*)ctx->scratch.get("solve_x", (size_t)R * nsp * 16);
    for (int r = 0; r < R; r++) {
      const double* din = stage_in(ctx, "canon_in", b + 2 * nsp * (r0 + r), nsp, loc);
      launch_spinor_from_canon(g, PREC_F64, bf + 2 * nsp * r, nullptr, din, ctx->stream);
    }
    OuterResult o = outer_fgmres(ctx, xf, bf, mu, R);
    for (int r = 0; r < R; r++) {
      double* dout = stage_out(ctx, "canon_out", x + 2 * nsp * (r0 + r), nsp, loc);
      launch_spinor_to_canon(g, PREC_F64, xf + 2 * nsp * r, nullptr, dout, ctx->stream);
      unstage_out(ctx, x + 2 * nsp * (r0 + r), dout, nsp, loc);
    }
    acc.iters = o.iters > acc.iters ? o.iters : acc.iters;
    acc.restarts = o.restarts > acc.restarts ? o.restarts : acc.restarts;
    for (double v : o.relres) acc.max_relres = v > acc.max_relres ? v : acc.max_relres;
    all_conv = all_conv && o.converged;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  check_tc_all(ctx);
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
  if (ok && ctx->p.n_levels == 3) {  // level-1 test vectors: nv1, block[1], then nv1 level-1 vectors (FP32)
    const size_t b1 = (size_t)ctx->a1.nv * ctx->c1.Nc * ctx->c1.n * sizeof(float2);
    std::vector<char> h1(b1);
    CK(cudaMemcpy(h1.data(), ctx->a1.tv.p, b1, cudaMemcpyDeviceToHost));
    int h2[5] = {ctx->a1.nv, ctx->p.block[1][0], ctx->p.block[1][1], ctx->p.block[1][2], ctx->p.block[1][3]};
    ok = fwrite(h2, sizeof(int), 5, f) == 5 && fwrite(h1.data(), 1, b1, f) == b1;
  }
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
  std::vector<char> h1;
  if (ok && ctx->p.n_levels == 3) {
    int h2[5];
    ok = fread(h2, sizeof(int), 5, f) == 5 && h2[0] == ctx->p.nv[1];
    for (int m = 0; ok && m < 4; m++) ok = h2[1 + m] == ctx->p.block[1][m];
    if (ok) {
      const size_t b1 = (size_t)h2[0] * ctx->g.Nb * 2 * hdr[8] * sizeof(float2);
      h1.resize(b1);
      ok = fread(h1.data(), 1, b1, f) == b1;
    }
  }
  fclose(f);
  if (!ok) throw Error(DDTM_ERR_ARG, "truncated setup file, or its level-1 part does not match the parameters");
  ctx->nv0 = hdr[8];
  ctx->tv0.ensure(bytes);
  CK(cudaMemcpyAsync(ctx->tv0.p, host.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
  build_hierarchy(ctx);
  if (ctx->p.n_levels == 3) {
    ctx->a1.nv = ctx->p.nv[1];
    ctx->a1.tv.ensure(h1.size());
    CK(cudaMemcpyAsync(ctx->a1.tv.p, h1.data(), h1.size(), cudaMemcpyHostToDevice, ctx->stream));
    build_hierarchy1(ctx);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->setup_mu = mu;
  ctx->setup_done = true;
  API_END(ctx)
}

}  // extern "C"

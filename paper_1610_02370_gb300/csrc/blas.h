// Host interface of the Krylov vector kernels (blas.cu).
//
// A "vector set" holds R right-hand sides of n complex entries each, either
// interleaved (element (e, r) at e * R + r: coarse vectors) or separate
// (element (e, r) at r * n + e: fine fields).  Type tags: 0 = double2 (FP64
// complex), 1 = float2 (FP32 complex), 2 = __half2 (FP16 complex storage,
// FP32 arithmetic; paired with FP32 sets only).  A basis of nvec sets lies at
// V + j*ldv (ldv in complex elements).  Inner products sum per thread in the
// operands' arithmetic precision (FP32 for FP32 / FP16 sets, FP64 otherwise),
// within a CTA in FP64 (generic kernels) or FP32 (pair kernels), and across
// CTAs in FP64, always in a fixed order (deterministic).
// Interleaved FP32 sets with an even number of right-hand sides use kernels
// that read 16-byte pairs of right-hand sides.  Results that come back to the
// host synchronise the stream; coefficients travel through a pinned ring of
// buffers guarded by events, so no call blocks on a copy.
#pragma once

#include <vector>

#include "ddtm_internal.h"

namespace ddtm {

struct VSet {
  void* p;
  int type;     // 0 double2, 1 float2, 2 __half2
  size_t n;     // complex entries per right-hand side
  int R;        // right-hand sides
  bool inter;   // interleaved (true) or separate (false)
};

struct Blas {
  cudaStream_t st;
  ScratchPool* pool;
  CoefRing* ring;
  Blas(cudaStream_t s, ScratchPool* pool, CoefRing* ring = nullptr);
  // out[j * R + r] = <V_j(., r), w(., r)> for j < nvec (host result)
  void dots(const VSet& V, size_t ldv, int nvec, const VSet& w, double2* out_host);
  // per-rhs squared norms (host result)
  void norms2(const VSet& a, double* out_host);
  // w(., r) += sign * sum_j coef[j * R + r] V_j(., r); with norms2_host != null
  // also returns ||w(., r)||^2 of the result
  void maxpy(const VSet& w, const VSet& V, size_t ldv, int nvec, const double2* coef_host, double sign,
             double* norms2_host);
  // y(., r) = a[r] x(., r) + b[r] y(., r); a zero coefficient skips reading its operand
  void axpby(const double2* a_host, const VSet& x, const double2* b_host, const VSet& y);

  // device-result variants: no host synchronisation, coefficients and results
  // stay in device memory (layouts as above)
  void dots_dev(const VSet& V, size_t ldv, int nvec, const VSet& w, double2* out_dev);
  void maxpy_dev(const VSet& w, const VSet& V, size_t ldv, int nvec, const double2* coef_dev, double sign,
                 double2* norms2_dev);
  // y(., r) = a[r] x(., r), a in device memory
  void scale_dev(const double2* a_dev, const VSet& x, const VSet& y);

  // single-vector conveniences (R = 1)
  double norm2(const void* a, int t, size_t n);
  void axpby(double2 a, const void* x, int tx, double2 b, void* y, int ty, size_t n);
};

// Arnoldi bookkeeping on the device for R lockstep GMRES systems (Givens
// rotations as in the host code: G = [[conj(c), conj(s)], [-s, c]]).
// State per system r: H[(r*(m+1) + i)*m + j], cs/sn[r*m + i], g[r*(m+1) + i].
struct ArnoldiDev {
  double2 *H, *cs, *sn, *g;
  double* bn;      // ||b_r||
  double* est;     // residual estimate / ||b_r||
  double2* scale;  // 1 / norm for the next basis vector (0 if the norm vanished)
  int m, R;
};
// start of a cycle from the squared residual norms nr2[r].x
void launch_arnoldi_start(const ArnoldiDev& a, const double2* nr2, cudaStream_t st);
// column j from the Gram-Schmidt coefficients h (+ h2 if non-null), [i*R + r],
// and the squared norm of the orthogonalised vector hn2[r].x
// fp32: rotations in FP32 arithmetic (state kept in FP64), for loose tolerances
void launch_arnoldi_step(const ArnoldiDev& a, int j, const double2* h, const double2* h2, const double2* hn2,
                         cudaStream_t st, bool fp32);
// y[i*R + r] from the triangular systems of the first k columns
void launch_arnoldi_solve(const ArnoldiDev& a, int k, double2* y, cudaStream_t st);

void launch_field_convert(const FineGeom& g, int pin, const void* in, const float* inn, int pout, void* out, float* outn,
                          cudaStream_t st);

}  // namespace ddtm

// The twisted-mass clover Wilson-Dirac operator D(mu) = D_W + i mu Gamma5
// (Sec. 2.1 of arXiv:1610.02370) on the internal even-odd block layout.
//
// * k_clover_build: the site term (m+4) I - c_sw/32 sum_{mu,nu} (gamma_mu
//   gamma_nu) x (Q_mu_nu - Q_nu_mu) from the four plaquette leaves Q_mu_nu of
//   Sec. 2.1, in FP64, once per gauge field.  With Q_nu_mu = Q_mu_nu^dagger the
//   sum is -c_sw/16 sum_{mu<nu} (gamma_mu gamma_nu) x F_mu_nu, F = Q - Q^dagger.
//   In the chiral basis every gamma_mu gamma_nu (mu != nu) is block diagonal in
//   chirality, so the site term is two Hermitian 6x6 blocks per site.
// * k_site_inverse: per even site and chirality h the inverse of
//   S_h + i mu_h (mu_0 = mu, mu_1 = -mu), by Gauss-Jordan elimination with
//   partial pivoting in FP64 (used by the even-odd block solves of SAP).
// * k_dslash: one thread per site; 8 neighbour half-spinor hops, clover and
//   twist; storage FP64 / FP32 / FP16 (per-site scaled spinors).
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"

namespace ddtm {

// 2x2 spin blocks of gamma_mu gamma_nu, pair p over (0,1),(0,2),(0,3),(1,2),(1,3),(2,3),
// chirality h: c_gg[((p*2 + h)*2 + s)*2 + t]
__constant__ double2 c_gg[6 * 2 * 2 * 2];
static bool gg_ready = false;

typedef cplx<double> zd;

static void host_gammas(zd g[4][4][4]) {
  for (int m = 0; m < 4; m++)
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) g[m][i][j] = zd(0, 0);
  // gamma_0 = [[0, 1], [1, 0]]
  for (int i = 0; i < 2; i++) { g[0][i][i + 2] = zd(1, 0); g[0][i + 2][i] = zd(1, 0); }
  // Pauli matrices
  zd s[3][2][2] = {{{zd(0, 0), zd(1, 0)}, {zd(1, 0), zd(0, 0)}},
                   {{zd(0, 0), zd(0, -1)}, {zd(0, 1), zd(0, 0)}},
                   {{zd(1, 0), zd(0, 0)}, {zd(0, 0), zd(-1, 0)}}};
  for (int k = 0; k < 3; k++)
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        g[k + 1][i][j + 2] = times_i(s[k][i][j]);         // i s_k
        g[k + 1][i + 2][j] = times_minus_i(s[k][i][j]);   // -i s_k
      }
}

static void upload_gg() {
  if (gg_ready) return;
  zd g[4][4][4];
  host_gammas(g);
  double2 h[48];
  int p = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++, p++) {
      zd prod[4][4];
      for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
          zd acc(0, 0);
          for (int k = 0; k < 4; k++) cmac(acc, g[mu][i][k], g[nu][k][j]);
          prod[i][j] = acc;
        }
      for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++)
          if ((i < 2) != (j < 2) && (prod[i][j].re != 0 || prod[i][j].im != 0))
            throw Error(DDTM_ERR_CUDA, "internal: gamma_mu gamma_nu not chirality block diagonal");
      for (int hh = 0; hh < 2; hh++)
        for (int s = 0; s < 2; s++)
          for (int t = 0; t < 2; t++) {
            zd v = prod[2 * hh + s][2 * hh + t];
            h[((p * 2 + hh) * 2 + s) * 2 + t] = make_double2(v.re, v.im);
          }
    }
  CK(cudaMemcpyToSymbol(c_gg, h, sizeof(h)));
  gg_ready = true;
}

// ---- 3x3 complex matrices (FP64) for the clover leaves -----------------------
struct M3 { zd a[9]; };

__device__ __forceinline__ M3 m3_load(const double2* U, size_t site, int mu) {
  M3 m;
  const double2* p = U + (site * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; k++) { double2 v = __ldg(p + k); m.a[k] = zd(v.x, v.y); }
  return m;
}
// op(A) op(B) with A^dagger / B^dagger selectable
__device__ __forceinline__ M3 m3_mul(const M3& A, bool da, const M3& B, bool db) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      zd acc(0, 0);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        zd a = da ? conj(A.a[k * 3 + i]) : A.a[i * 3 + k];
        zd b = db ? conj(B.a[j * 3 + k]) : B.a[k * 3 + j];
        cmac(acc, a, b);
      }
      C.a[i * 3 + j] = acc;
    }
  return C;
}

struct Lat { int L[4]; };

__device__ __forceinline__ size_t site_at(const Lat& l, const int c[4], int d1, int s1, int d2, int s2) {
  int x[4] = {c[0], c[1], c[2], c[3]};
  if (d1 >= 0) x[d1] = (x[d1] + s1 + l.L[d1]) % l.L[d1];
  if (d2 >= 0) x[d2] = (x[d2] + s2 + l.L[d2]) % l.L[d2];
  return (((size_t)x[0] * l.L[3] + x[3]) * l.L[2] + x[2]) * l.L[1] + x[1];
}

// Q_mu_nu(x): the four leaves in the order printed in Sec. 2.1
__device__ M3 clover_leaves(const double2* U, const Lat& l, const int c[4], int mu, int nu) {
  size_t x = site_at(l, c, -1, 0, -1, 0);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
  M3 t = m3_mul(m3_load(U, x, mu), false, m3_load(U, site_at(l, c, mu, 1, -1, 0), nu), false);
  t = m3_mul(t, false, m3_load(U, site_at(l, c, nu, 1, -1, 0), mu), true);
  M3 Q = m3_mul(t, false, m3_load(U, x, nu), true);
  // leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
  t = m3_mul(m3_load(U, x, nu), false, m3_load(U, site_at(l, c, mu, -1, nu, 1), mu), true);
  t = m3_mul(t, false, m3_load(U, site_at(l, c, mu, -1, -1, 0), nu), true);
  t = m3_mul(t, false, m3_load(U, site_at(l, c, mu, -1, -1, 0), mu), false);
#pragma unroll
  for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + t.a[k];
  // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
  t = m3_mul(m3_load(U, site_at(l, c, mu, -1, -1, 0), mu), true, m3_load(U, site_at(l, c, mu, -1, nu, -1), nu), true);
  t = m3_mul(t, false, m3_load(U, site_at(l, c, mu, -1, nu, -1), mu), false);
  t = m3_mul(t, false, m3_load(U, site_at(l, c, nu, -1, -1, 0), nu), false);
#pragma unroll
  for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + t.a[k];
  // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
  t = m3_mul(m3_load(U, site_at(l, c, nu, -1, -1, 0), nu), true, m3_load(U, site_at(l, c, nu, -1, -1, 0), mu), false);
  t = m3_mul(t, false, m3_load(U, site_at(l, c, nu, -1, mu, 1), nu), false);
  t = m3_mul(t, false, m3_load(U, x, mu), true);
#pragma unroll
  for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + t.a[k];
  return Q;
}

struct BlockMap {
  int b[4], NB[4];
  int Vb;
  const uint32_t* loc_coord;
};

__global__ void k_clover_build(double2* __restrict__ out, const double2* __restrict__ U, Lat l, BlockMap m,
                               double m4, double csw, long V) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int blk = (int)(s / m.Vb), loc = (int)(s - (long)blk * m.Vb);
  int B[4], r = blk;
  B[1] = r % m.NB[1]; r /= m.NB[1];
  B[2] = r % m.NB[2]; r /= m.NB[2];
  B[3] = r % m.NB[3];
  B[0] = r / m.NB[3];
  uint32_t lc = m.loc_coord[loc];
  int c[4] = {B[0] * m.b[0] + (int)(lc & 255), B[1] * m.b[1] + (int)((lc >> 8) & 255),
              B[2] * m.b[2] + (int)((lc >> 16) & 255), B[3] * m.b[3] + (int)((lc >> 24) & 255)};
  zd S[2][6][6];
#pragma unroll
  for (int h = 0; h < 2; h++)
    for (int i = 0; i < 6; i++)
      for (int j = 0; j < 6; j++) S[h][i][j] = zd(i == j ? m4 : 0.0, 0.0);
  int p = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++, p++) {
      M3 Q = clover_leaves(U, l, c, mu, nu);
      zd F[9];
#pragma unroll
      for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) F[a * 3 + b] = Q.a[a * 3 + b] - conj(Q.a[b * 3 + a]);
      for (int h = 0; h < 2; h++)
        for (int s2 = 0; s2 < 2; s2++)
          for (int t2 = 0; t2 < 2; t2++) {
            double2 gv = c_gg[((p * 2 + h) * 2 + s2) * 2 + t2];
            zd g(gv.x * (-csw / 16.0), gv.y * (-csw / 16.0));
            for (int a = 0; a < 3; a++)
              for (int b = 0; b < 3; b++) cmac(S[h][s2 * 3 + a][t2 * 3 + b], g, F[a * 3 + b]);
          }
    }
  // pack: diagonal reals, then the upper triangle
  for (int h = 0; h < 2; h++) {
    for (int k = 0; k < 3; k++)
      out[((size_t)blk * 36 + h * 18 + k) * m.Vb + loc] = make_double2(S[h][2 * k][2 * k].re, S[h][2 * k + 1][2 * k + 1].re);
    int slot = 3;
    for (int i = 0; i < 6; i++)
      for (int j = i + 1; j < 6; j++, slot++)
        out[((size_t)blk * 36 + h * 18 + slot) * m.Vb + loc] = make_double2(S[h][i][j].re, S[h][i][j].im);
  }
}

void launch_clover_build(const FineGeom& g, double* clov, const double* Ucanon, double m_plus_4, double csw,
                         cudaStream_t s) {
  ScopedTimer timer_("clover_build", s);
  upload_gg();
  Lat l;
  BlockMap m;
  for (int i = 0; i < 4; i++) { l.L[i] = g.L[i]; m.b[i] = g.b[i]; m.NB[i] = g.NB[i]; }
  m.Vb = g.Vb;
  m.loc_coord = g.loc_coord.as<uint32_t>();
  k_clover_build<<<(unsigned)((g.V + 63) / 64), 64, 0, s>>>((double2*)clov, (const double2*)Ucanon, l, m, m_plus_4,
                                                           csw, g.V);
  CKL("clover_build");
}

// ---- inverse of the site-local operator on even sites ------------------------
template <int P>
__global__ void k_site_inverse(typename Prec<P>::store2* __restrict__ out, const double2* __restrict__ clov,
                               int Vb, int Nb, double mu) {
  int Vh = Vb / 2;
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)Nb * Vh * 2) return;
  int h = (int)(t & 1);
  long sh = t >> 1;
  int blk = (int)(sh / Vh), loc = (int)(sh - (long)blk * Vh);  // even sites: loc < Vh
  zd A[6][6], X[6][6];
  const double2* p = clov + (size_t)blk * 36 * Vb + loc;
  for (int k = 0; k < 3; k++) {
    double2 d = p[(size_t)(h * 18 + k) * Vb];
    A[2 * k][2 * k] = zd(d.x, 0);
    A[2 * k + 1][2 * k + 1] = zd(d.y, 0);
  }
  int slot = 3;
  for (int i = 0; i < 6; i++)
    for (int j = i + 1; j < 6; j++, slot++) {
      double2 u = p[(size_t)(h * 18 + slot) * Vb];
      A[i][j] = zd(u.x, u.y);
      A[j][i] = zd(u.x, -u.y);
    }
  double mh = h == 0 ? mu : -mu;
  for (int i = 0; i < 6; i++) {
    A[i][i].im += mh;
    for (int j = 0; j < 6; j++) X[i][j] = zd(i == j ? 1.0 : 0.0, 0.0);
  }
  for (int col = 0; col < 6; col++) {
    int piv = col;
    double best = norm2(A[col][col]);
    for (int r = col + 1; r < 6; r++)
      if (norm2(A[r][col]) > best) { best = norm2(A[r][col]); piv = r; }
    if (piv != col)
      for (int j = 0; j < 6; j++) {
        zd tmp = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = tmp;
        tmp = X[col][j]; X[col][j] = X[piv][j]; X[piv][j] = tmp;
      }
    zd d = A[col][col];
    double dn = norm2(d);
    zd inv(d.re / dn, -d.im / dn);
    for (int j = 0; j < 6; j++) { A[col][j] = A[col][j] * inv; X[col][j] = X[col][j] * inv; }
    for (int r = 0; r < 6; r++) {
      if (r == col) continue;
      zd f = A[r][col];
      for (int j = 0; j < 6; j++) {
        A[r][j] = A[r][j] - f * A[col][j];
        X[r][j] = X[r][j] - f * X[col][j];
      }
    }
  }
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) {
      cplx<typename Prec<P>::real> v((typename Prec<P>::real)X[i][j].re, (typename Prec<P>::real)X[i][j].im);
      st(out + ((size_t)blk * 72 + h * 36 + i * 6 + j) * Vh + loc, v);
    }
}

void launch_site_inverse(const FineGeom& g, int prec, void* out, const double* clov64, double mu, cudaStream_t s) {
  ScopedTimer timer_("site_inverse", s);
  long n = (long)g.Nb * g.Vb;  // Nb * Vh * 2
  unsigned grid = (unsigned)((n + 127) / 128);
  if (prec == PREC_F64) k_site_inverse<PREC_F64><<<grid, 128, 0, s>>>((double2*)out, (const double2*)clov64, g.Vb, g.Nb, mu);
  else if (prec == PREC_F32) k_site_inverse<PREC_F32><<<grid, 128, 0, s>>>((float2*)out, (const double2*)clov64, g.Vb, g.Nb, mu);
  else k_site_inverse<PREC_F16><<<grid, 128, 0, s>>>((__half2*)out, (const double2*)clov64, g.Vb, g.Nb, mu);
  CKL("site_inverse");
}

// ---- the stencil -----------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_dslash(Spinor<P> y, Spinor<P> x, Links<P> U, Clover<P> C, Geo g,
                                                typename Prec<P>::real mu) {
  typedef typename Prec<P>::real R;
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)g.Vb * g.Nb) return;
  int blk = (int)(s / g.Vb), loc = (int)(s - (long)blk * g.Vb);
  cplx<R> acc[12];
#pragma unroll
  for (int c = 0; c < 12; c++) acc[c] = cplx<R>(0, 0);
#pragma unroll
  for (int mu_ = 0; mu_ < 4; mu_++) {
#pragma unroll
    for (int dir = 0; dir < 2; dir++) {
      bool fwd = dir == 0;
      Nbr n = neighbour(g, blk, loc, 2 * mu_ + dir);
      cplx<R> h[6], w[6], u[9];
      {
        cplx<R> p[12];
        x.load(n.blk, n.loc, p);
        project<R>(mu_, fwd, p, h);
      }
      if (fwd) {
        U.load(blk, loc, mu_, u);
        mul_U<R>(u, h, w);
      } else {
        U.load(n.blk, n.loc, mu_, u);
        mul_Udag<R>(u, h, w);
      }
      if (n.flip) {
#pragma unroll
        for (int k = 0; k < 6; k++) w[k] = -w[k];
      }
      reconstruct<R>(mu_, fwd, w, acc);
    }
  }
  cplx<R> in[12], out[12];
  x.load(blk, loc, in);
  C.apply(blk, loc, in, out);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    cplx<R> tw = times_i(in[c]);
    R m = c < 6 ? mu : -mu;
    out[c] = out[c] + m * tw + R(-0.5) * acc[c];
  }
  y.store(blk, loc, out);
}

// ---- the stencil on whole lattice blocks -------------------------------------------------
// One CTA per lattice block of VB sites (a compile-time size, so every
// component offset inside the block is an immediate), one thread per site,
// nrhs right-hand sides one after another.  For each right-hand side the
// block's x is read once from HBM (coalesced, one component per warp load),
// converted to FP32 with its per-site scale and staged in shared memory; the
// hops that stay inside the block (3/4 of them for 4^4 blocks) read their
// neighbour there, the hops that leave it read the neighbour block in global
// memory.  Links and the clover term of the block are read through the
// read-only cache with immediate offsets; with several right-hand sides the
// CTA re-reads them from L1/L2, so HBM sees them once per launch.
template <int P, int VB>
__global__ void __launch_bounds__(VB, 3)
    k_dslash_blk(Spinor<P> y, Spinor<P> x, Links<P> U, Clover<P> C, Geo g, float mu, int nrhs, size_t fstride,
                 long V) {
  typedef typename Prec<P>::store2 S;
  __shared__ float2 xs[12 * VB];
  const int blk = blockIdx.x, loc = threadIdx.x;
  const S* ub = U.d + (size_t)blk * 36 * VB;
  for (int r = 0; r < nrhs; r++) {
    Spinor<P> xr = x, yr = y;
    xr.d += (size_t)r * fstride;
    yr.d += (size_t)r * fstride;
    if (Prec<P>::scaled) {
      xr.nrm += (size_t)r * V;
      yr.nrm += (size_t)r * V;
    }
    {
      cplx<float> in[12];
      xr.load(blk, loc, in);
#pragma unroll
      for (int c = 0; c < 12; c++) xs[c * VB + loc] = make_float2(in[c].re, in[c].im);
    }
    __syncthreads();
    cplx<float> acc[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = cplx<float>(0, 0);
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int mu_ = k >> 1;
      const bool fwd = (k & 1) == 0;
      const uint32_t e = __ldg(g.loc_nbr + k * VB + loc);
      const int nloc = e & 0xffff;
      const bool cross = (e >> 16) & 1;
      cplx<float> h[6], w[6], u[9];
      int nblk = blk;
      float sgn = 1.f;
      {
        cplx<float> p[12];
        if (!cross) {
#pragma unroll
          for (int c = 0; c < 12; c++) {
            float2 v = xs[c * VB + nloc];
            p[c] = cplx<float>(v.x, v.y);
          }
        } else {
          const int b = __ldg(g.blk_nbr + k * g.Nb + blk);
          nblk = b & 0x3fffffff;
          sgn = (b >> 30) & 1 ? -1.f : 1.f;
          xr.load(nblk, nloc, p);
        }
        project<float>(mu_, fwd, p, h);
      }
      const S* ul = (fwd ? ub : U.d + (size_t)nblk * 36 * VB) + mu_ * 9 * VB + (fwd ? loc : nloc);
#pragma unroll
      for (int q = 0; q < 9; q++) u[q] = ld(ul + q * VB);
      if (fwd) mul_U<float>(u, h, w);
      else mul_Udag<float>(u, h, w);
#pragma unroll
      for (int q = 0; q < 6; q++) w[q] = sgn * w[q];
      reconstruct<float>(mu_, fwd, w, acc);
    }
    cplx<float> in[12], out[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
      float2 v = xs[c * VB + loc];
      in[c] = cplx<float>(v.x, v.y);
    }
    C.apply(blk, loc, in, out);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      const float m = c < 6 ? mu : -mu;
      out[c] = out[c] + m * times_i(in[c]) + (-0.5f) * acc[c];
    }
    yr.store(blk, loc, out);
    __syncthreads();  // xs is overwritten by the next right-hand side
  }
}

static Geo make_geo(const FineGeom& g) {
  Geo q;
  q.Vb = g.Vb;
  q.Nb = g.Nb;
  q.loc_nbr = g.loc_nbr.as<uint32_t>();
  q.blk_nbr = g.blk_nbr.as<int>();
  return q;
}

// Block kernels exist for 4^4 blocks (VB = 256) in FP32 and FP16 storage.
static bool dslash_blk_ok(const FineGeom& g, int prec) { return prec != PREC_F64 && g.Vb == 256; }

template <int P>
static void dslash_blk_t(const FineGeom& g, void* y, float* ynrm, const void* x, const float* xnrm, const void* links,
                         const void* clover, double mu, int nrhs, cudaStream_t s) {
  typedef typename Prec<P>::store2 S;
  Spinor<P> Y{(S*)y, ynrm, g.Vb}, X{(S*)x, (float*)xnrm, g.Vb};
  k_dslash_blk<P, 256><<<g.Nb, 256, 0, s>>>(Y, X, Links<P>{(const S*)links, g.Vb}, Clover<P>{(const S*)clover, g.Vb},
                                             make_geo(g), (float)mu, nrhs, (size_t)g.V * 12, g.V);
  CKL("dslash_blk");
}

// y = D(mu) x for nrhs right-hand sides at stride 12 V (store2 elements; FP16
// scales at stride V): one launch for all of them with the block kernel, else
// one launch per right-hand side.
void launch_dslash_multi(const FineGeom& g, int prec, void* y, float* ynrm, const void* x, const float* xnrm,
                         const void* links, const void* clover, double mu, int nrhs, cudaStream_t s) {
  if (nrhs <= 0) return;
  if (!dslash_blk_ok(g, prec)) {
    const size_t fb = (size_t)g.V * 12 * (prec == PREC_F64 ? 16 : prec == PREC_F32 ? 8 : 4);
    for (int r = 0; r < nrhs; r++)
      launch_dslash(g, prec, (char*)y + r * fb, ynrm ? ynrm + (size_t)r * g.V : nullptr, (const char*)x + r * fb,
                    xnrm ? xnrm + (size_t)r * g.V : nullptr, links, clover, mu, s);
    return;
  }
  ScopedTimer timer_(prec == PREC_F32 ? "dslash_f32" : "dslash_f16", s, nrhs);
  if (prec == PREC_F32) dslash_blk_t<PREC_F32>(g, y, ynrm, x, xnrm, links, clover, mu, nrhs, s);
  else dslash_blk_t<PREC_F16>(g, y, ynrm, x, xnrm, links, clover, mu, nrhs, s);
}

void launch_dslash(const FineGeom& g, int prec, void* y, float* ynrm, const void* x, const float* xnrm,
                   const void* links, const void* clover, double mu, cudaStream_t s) {
  if (dslash_blk_ok(g, prec)) {
    launch_dslash_multi(g, prec, y, ynrm, x, xnrm, links, clover, mu, 1, s);
    return;
  }
  ScopedTimer timer_(prec == PREC_F64 ? "dslash_f64" : prec == PREC_F32 ? "dslash_f32" : "dslash_f16", s);
  Geo q = make_geo(g);
  unsigned grid = (unsigned)((g.V + 127) / 128);
  if (prec == PREC_F64) {
    Spinor<PREC_F64> Y{(double2*)y, nullptr, g.Vb}, X{(double2*)x, nullptr, g.Vb};
    k_dslash<PREC_F64><<<grid, 128, 0, s>>>(Y, X, Links<PREC_F64>{(const double2*)links, g.Vb},
                                            Clover<PREC_F64>{(const double2*)clover, g.Vb}, q, mu);
  } else if (prec == PREC_F32) {
    Spinor<PREC_F32> Y{(float2*)y, nullptr, g.Vb}, X{(float2*)x, nullptr, g.Vb};
    k_dslash<PREC_F32><<<grid, 128, 0, s>>>(Y, X, Links<PREC_F32>{(const float2*)links, g.Vb},
                                            Clover<PREC_F32>{(const float2*)clover, g.Vb}, q, (float)mu);
  } else {
    Spinor<PREC_F16> Y{(__half2*)y, ynrm, g.Vb}, X{(__half2*)x, (float*)xnrm, g.Vb};
    k_dslash<PREC_F16><<<grid, 128, 0, s>>>(Y, X, Links<PREC_F16>{(const __half2*)links, g.Vb},
                                            Clover<PREC_F16>{(const __half2*)clover, g.Vb}, q, (float)mu);
  }
  CKL("dslash");
}

}  // namespace ddtm

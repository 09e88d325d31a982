// Red-black multiplicative SAP smoother (Sec. 2.4) with even-odd reduced
// block solves by minimal residual (Sec. 2.4, 2.5).
//
// One launch is one half-sweep over the blocks of one colour; one CTA owns one
// block.  Blocks of one colour never touch, so CTAs are independent: each reads
// x on its own block and on the neighbouring blocks of the other colour and
// writes x only on its own block.  Per block B:
//   r     = b - D(mu) x                 on B (full stencil, neighbours in HBM)
//   rhat  = r_o - A_oe A_ee^-1 r_e      (A = D_BB + i mu Gamma5, hops leaving B dropped)
//   e_o   = nmr MR steps on A_hat e_o = rhat from 0,
//           A_hat = A_oo - A_oe A_ee^-1 A_eo,  alpha = <p, rho> / <p, p>
//   e_e   = A_ee^-1 (r_e - A_eo e_o)
//   x_B  += e
// A_ee^-1 is the precomputed inverse of the site term + i mu gamma5 on even
// sites.  Vectors of the block solve live in shared memory as [12][Vh]; inner
// products are reduced per CTA in a fixed order (deterministic).
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"
#include "stencil.cuh"

namespace ddtm {

template <typename R>
struct SapArgs {
  const int* blocks;       // blocks of this colour
  const int* zero_blocks;  // first sweep from x = 0: blocks of the other colour to clear
  int zero_x;              // x is implicitly zero on entry
  int nmr;
  R mu;
  size_t fstride;          // store2 elements between right-hand sides (12 V)
  long V;                  // sites (stride of the FP16 scales between right-hand sides)
};

// sum over the CTA of three reals; every thread receives the totals
template <typename R>
__device__ __forceinline__ void cta_sum3(R& a, R& b, R& c, R* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[3 * w] = a;
    red[3 * w + 1] = b;
    red[3 * w + 2] = c;
  }
  __syncthreads();
  a = b = c = 0;
  for (int i = 0; i < nw; i++) {
    a += red[3 * i];
    b += red[3 * i + 1];
    c += red[3 * i + 2];
  }
}

template <int P>
__global__ void __launch_bounds__(128, P == PREC_F64 ? 2 : 4) k_sap_half(Spinor<P> x, Spinor<P> b, Links<P> U, Clover<P> C, SiteInv<P> Ainv, Geo g,
                           SapArgs<typename Prec<P>::real> a) {
  typedef typename Prec<P>::real R;
  typedef cplx<R> Z;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vh = g.Vb / 2;
  Z* rho = reinterpret_cast<Z*>(smem_raw);  // odd sites: residual of the reduced system
  Z* te = rho + 12 * Vh;                    // even sites: intermediate
  Z* re = te + 12 * Vh;                     // even sites: block residual r_e
  Z* eo = re + 12 * Vh;                     // odd sites: correction e_o
  R* red = reinterpret_cast<R*>(eo + 12 * Vh);

  // grid: x = right-hand side, y = block of this colour
  const int rhs = blockIdx.x;
  x.d += (size_t)rhs * a.fstride;
  b.d += (size_t)rhs * a.fstride;
  if (x.nrm) x.nrm += (size_t)rhs * a.V;
  if (b.nrm) b.nrm += (size_t)rhs * a.V;
  const int blk = a.blocks[blockIdx.y];
  const int i = threadIdx.x;
  const bool act = i < Vh;
  const int le = i, lo = Vh + i;  // this thread's even and odd site

  if (a.zero_x && act) {  // clear one block of the other colour (x = 0 start)
    Z zero[12];
#pragma unroll
    for (int c = 0; c < 12; c++) zero[c] = Z(0, 0);
    int zb = a.zero_blocks[blockIdx.y];
    x.store(zb, le, zero);
    x.store(zb, lo, zero);
  }

  // 1. block residual r = b - D x on both parities
  if (act) {
    Z bb[12], dx[12];
    b.load(blk, le, bb);
    if (!a.zero_x) {
      dslash_site<P, 1>(x, U, C, g, a.mu, blk, le, dx);
#pragma unroll
      for (int c = 0; c < 12; c++) bb[c] = bb[c] - dx[c];
    }
#pragma unroll
    for (int c = 0; c < 12; c++) re[c * Vh + i] = bb[c];
    Z t[12];
    Ainv.apply(blk, le, bb, t);
#pragma unroll
    for (int c = 0; c < 12; c++) te[c * Vh + i] = t[c];
    b.load(blk, lo, bb);
    if (!a.zero_x) {
      dslash_site<P, 1>(x, U, C, g, a.mu, blk, lo, dx);
#pragma unroll
      for (int c = 0; c < 12; c++) bb[c] = bb[c] - dx[c];
    }
#pragma unroll
    for (int c = 0; c < 12; c++) {
      rho[c * Vh + i] = bb[c];
      eo[c * Vh + i] = Z(0, 0);
    }
  }
  __syncthreads();
  // 2. rhat = r_o - H_oe A_ee^-1 r_e
  if (act) {
    Z h[12];
    hop_block<P, R>(te, Vh, U, g, blk, lo, h);
#pragma unroll
    for (int c = 0; c < 12; c++) rho[c * Vh + i] = rho[c * Vh + i] - h[c];
  }
  __syncthreads();
  // 3. MR on the reduced block system
  for (int k = 0; k < a.nmr; k++) {
    if (act) {  // te = A_ee^-1 H_eo rho
      Z h[12], t[12];
      hop_block<P, R>(rho, Vh, U, g, blk, le, h);
      Ainv.apply(blk, le, h, t);
#pragma unroll
      for (int c = 0; c < 12; c++) te[c * Vh + i] = t[c];
    }
    __syncthreads();
    Z p[12];
    R pr_re = 0, pr_im = 0, pp = 0;
    if (act) {  // p = A_oo rho - H_oe te
      Z r[12], h[12];
#pragma unroll
      for (int c = 0; c < 12; c++) r[c] = rho[c * Vh + i];
      C.apply(blk, lo, r, p);
#pragma unroll
      for (int c = 0; c < 12; c++) {
        R m = c < 6 ? a.mu : -a.mu;
        p[c] = p[c] + m * times_i(r[c]);
      }
      hop_block<P, R>(te, Vh, U, g, blk, lo, h);
#pragma unroll
      for (int c = 0; c < 12; c++) {
        p[c] = p[c] - h[c];
        pr_re += p[c].re * r[c].re + p[c].im * r[c].im;  // <p, rho> = sum conj(p) rho
        pr_im += p[c].re * r[c].im - p[c].im * r[c].re;
        pp += norm2(p[c]);
      }
    }
    cta_sum3<R>(pr_re, pr_im, pp, red);
    Z alpha = pp > 0 ? Z(pr_re / pp, pr_im / pp) : Z(0, 0);
    if (act) {
#pragma unroll
      for (int c = 0; c < 12; c++) {
        Z r = rho[c * Vh + i];
        eo[c * Vh + i] = eo[c * Vh + i] + alpha * r;
        rho[c * Vh + i] = r - alpha * p[c];
      }
    }
    __syncthreads();
  }
  // 4. e_e = A_ee^-1 (r_e - H_eo e_o); 5. x_B += e
  if (act) {
    Z h[12], t[12], xv[12];
    hop_block<P, R>(eo, Vh, U, g, blk, le, h);
#pragma unroll
    for (int c = 0; c < 12; c++) h[c] = re[c * Vh + i] - h[c];
    Ainv.apply(blk, le, h, t);
    if (a.zero_x) {
      x.store(blk, le, t);
#pragma unroll
      for (int c = 0; c < 12; c++) xv[c] = eo[c * Vh + i];
      x.store(blk, lo, xv);
    } else {
      x.loadw(blk, le, xv);
#pragma unroll
      for (int c = 0; c < 12; c++) xv[c] = xv[c] + t[c];
      x.store(blk, le, xv);
      x.loadw(blk, lo, xv);
#pragma unroll
      for (int c = 0; c < 12; c++) xv[c] = xv[c] + eo[c * Vh + i];
      x.store(blk, lo, xv);
    }
  }
}

size_t sap_smem_bytes(int Vb, int prec) {
  size_t rb = prec == PREC_F64 ? 8 : 4;
  return 4 * 12 * (size_t)(Vb / 2) * 2 * rb + 3 * 32 * rb;
}

int sap_threads(int Vb) {
  int Vh = Vb / 2;
  return ((Vh + 31) / 32) * 32;
}

template <int P>
static void launch_sap_half_t(const FineGeom& g, void* x, float* xn, const void* b, const float* bn, const void* links,
                              const void* clover, const void* sinv, const int* blocks, const int* zero_blocks,
                              int nblocks, int zero_x, int nmr, double mu, int nrhs, cudaStream_t s) {
  typedef typename Prec<P>::store2 S;
  typedef typename Prec<P>::real R;
  Geo q{g.Vb, g.Nb, g.loc_nbr.as<uint32_t>(), g.blk_nbr.as<int>()};
  size_t smem = sap_smem_bytes(g.Vb, P);
  set_dynamic_smem((const void*)k_sap_half<P>, smem);
  // grid.y is at most 65535: on large lattices (e.g. 128 x 64^3 with 4^4 blocks, 65536 blocks per
  // colour) the blocks of the colour go in several launches, which is exact since they are independent
  for (int b0 = 0; b0 < nblocks; b0 += 65535) {
    const int nb = nblocks - b0 < 65535 ? nblocks - b0 : 65535;
    SapArgs<R> a{blocks + b0, zero_blocks + b0, zero_x, nmr, (R)mu, (size_t)g.V * 12, g.V};
    dim3 grid(nrhs, nb);
    k_sap_half<P><<<grid, sap_threads(g.Vb), smem, s>>>(
        Spinor<P>{(S*)x, xn, g.Vb}, Spinor<P>{(S*)b, (float*)bn, g.Vb}, Links<P>{(const S*)links, g.Vb},
        Clover<P>{(const S*)clover, g.Vb}, SiteInv<P>{(const S*)sinv, g.Vb / 2}, q, a);
    CKL("sap_half");
  }
}

void launch_sap_half(const FineGeom& g, int prec, void* x, float* xn, const void* b, const float* bn, const void* links,
                     const void* clover, const void* sinv, const int* blocks, const int* zero_blocks, int nblocks,
                     int zero_x, int nmr, double mu, int nrhs, cudaStream_t s) {
  ScopedTimer timer_(prec == PREC_F64 ? "sap_half_f64" : prec == PREC_F32 ? "sap_half_f32" : "sap_half_f16", s, nrhs);
  if (prec == PREC_F64)
    launch_sap_half_t<PREC_F64>(g, x, xn, b, bn, links, clover, sinv, blocks, zero_blocks, nblocks, zero_x, nmr, mu, nrhs, s);
  else if (prec == PREC_F32)
    launch_sap_half_t<PREC_F32>(g, x, xn, b, bn, links, clover, sinv, blocks, zero_blocks, nblocks, zero_x, nmr, mu, nrhs, s);
  else
    launch_sap_half_t<PREC_F16>(g, x, xn, b, bn, links, clover, sinv, blocks, zero_blocks, nblocks, zero_x, nmr, mu, nrhs, s);
}

}  // namespace ddtm

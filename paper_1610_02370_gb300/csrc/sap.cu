// Red-black multiplicative SAP smoother (Sec. 2.4) with even-odd reduced
// block solves by minimal residual (Sec. 2.4, 2.5).
//
// One launch is one half-sweep over the blocks of one colour; one CTA owns one
// block and RG right-hand sides of it (one group of threads per right-hand
// side, synchronised by its own named barrier), so the groups read the same
// links, clover entries and inverses at about the same time and all but the
// first are served by L1.  Blocks of one colour never touch, so CTAs are
// independent: each reads x on its own block and on the neighbouring blocks of
// the other colour and writes x only on its own block.  Per block B:
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
  int nrhs;                // right-hand sides of the batch
  const int* zero_blocks;  // first sweep from x = 0: blocks of the other colour to clear
  int zero_x;              // x is implicitly zero on entry
  int nmr;
  R mu;
  size_t fstride;          // store2 elements between right-hand sides (12 V)
  long V;                  // sites (stride of the FP16 scales between right-hand sides)
};

// shared memory of one right-hand-side group: four block vectors of 12 x Vh
// complex and the reduction slots, rounded to 16 bytes
template <typename R>
__host__ __device__ constexpr size_t sap_group_smem(int Vh) {
  return (4 * 12 * (size_t)Vh * 2 * sizeof(R) + 3 * 32 * sizeof(R) + 15) / 16 * 16;
}

// barrier of one right-hand-side group (gt threads, a multiple of 32): named
// barrier 1 + grp, or the whole CTA when it holds one group
template <int RG>
__device__ __forceinline__ void group_sync(int grp, int gt) {
  if (RG == 1) {
    __syncthreads();
    return;
  }
  switch (grp) {  // literal barrier ids, so the kernel reserves RG + 1 barriers, not all 16
    case 0: asm volatile("bar.sync 1, %0;" ::"r"(gt) : "memory"); break;
    case 1: asm volatile("bar.sync 2, %0;" ::"r"(gt) : "memory"); break;
    case 2: asm volatile("bar.sync 3, %0;" ::"r"(gt) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"r"(gt) : "memory"); break;
  }
}

// sum over the thread group (gt threads from thread grp * gt) of three reals;
// every thread of the group receives the totals
template <int RG, typename R>
__device__ __forceinline__ void group_sum3(R& a, R& b, R& c, R* red, int grp, int gt) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int w = (threadIdx.x - grp * gt) >> 5, nw = gt >> 5;
  group_sync<RG>(grp, gt);
  if ((threadIdx.x & 31) == 0) {
    red[3 * w] = a;
    red[3 * w + 1] = b;
    red[3 * w + 2] = c;
  }
  group_sync<RG>(grp, gt);
  a = b = c = 0;
  for (int i = 0; i < nw; i++) {
    a += red[3 * i];
    b += red[3 * i + 1];
    c += red[3 * i + 2];
  }
}

template <int P, int RG>
__global__ void __launch_bounds__(128 * RG, P == PREC_F64 ? 2 : 4 / RG)
    k_sap_half(Spinor<P> x, Spinor<P> b, Links<P> U, Clover<P> C, SiteInv<P> Ainv, Geo g,
               SapArgs<typename Prec<P>::real> a) {
  typedef typename Prec<P>::real R;
  typedef cplx<R> Z;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vh = g.Vb / 2;
  const int gt = blockDim.x / RG, grp = threadIdx.x / gt;  // group size and this thread's group
  // grid: x = group of RG right-hand sides, y = block of this colour
  const int rhs = blockIdx.x * RG + grp;
  if (rhs >= a.nrhs) return;  // a ragged last group: its barrier has no other members
  Z* rho = reinterpret_cast<Z*>(smem_raw + (size_t)grp * sap_group_smem<R>(Vh));  // odd sites: residual of the reduced system
  Z* te = rho + 12 * Vh;                    // even sites: intermediate
  Z* re = te + 12 * Vh;                     // even sites: block residual r_e
  Z* eo = re + 12 * Vh;                     // odd sites: correction e_o
  R* red = reinterpret_cast<R*>(eo + 12 * Vh);

  x.d += (size_t)rhs * a.fstride;
  b.d += (size_t)rhs * a.fstride;
  if (x.nrm) x.nrm += (size_t)rhs * a.V;
  if (b.nrm) b.nrm += (size_t)rhs * a.V;
  const int blk = a.blocks[blockIdx.y];
  const int i = threadIdx.x - grp * gt;
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
  group_sync<RG>(grp, gt);
  // 2. rhat = r_o - H_oe A_ee^-1 r_e
  if (act) {
    Z h[12];
    hop_block<P, R>(te, Vh, U, g, blk, lo, h);
#pragma unroll
    for (int c = 0; c < 12; c++) rho[c * Vh + i] = rho[c * Vh + i] - h[c];
  }
  group_sync<RG>(grp, gt);
  // 3. MR on the reduced block system
  for (int k = 0; k < a.nmr; k++) {
    if (act) {  // te = A_ee^-1 H_eo rho
      Z h[12], t[12];
      hop_block<P, R>(rho, Vh, U, g, blk, le, h);
      Ainv.apply(blk, le, h, t);
#pragma unroll
      for (int c = 0; c < 12; c++) te[c * Vh + i] = t[c];
    }
    group_sync<RG>(grp, gt);
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
    group_sum3<RG, R>(pr_re, pr_im, pp, red, grp, gt);
    Z alpha = pp > 0 ? Z(pr_re / pp, pr_im / pp) : Z(0, 0);
    if (act) {
#pragma unroll
      for (int c = 0; c < 12; c++) {
        Z r = rho[c * Vh + i];
        eo[c * Vh + i] = eo[c * Vh + i] + alpha * r;
        rho[c * Vh + i] = r - alpha * p[c];
      }
    }
    group_sync<RG>(grp, gt);
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
  return prec == PREC_F64 ? sap_group_smem<double>(Vb / 2) : sap_group_smem<float>(Vb / 2);
}

int sap_threads(int Vb) {
  int Vh = Vb / 2;
  return ((Vh + 31) / 32) * 32;
}

template <int P, int RG>
static void launch_sap_rg(const FineGeom& g, void* x, float* xn, const void* b, const float* bn, const void* links,
                          const void* clover, const void* sinv, const int* blocks, const int* zero_blocks, int nblocks,
                          int zero_x, int nmr, double mu, int nrhs, cudaStream_t s) {
  typedef typename Prec<P>::store2 S;
  typedef typename Prec<P>::real R;
  Geo q{g.Vb, g.Nb, g.loc_nbr.as<uint32_t>(), g.blk_nbr.as<int>()};
  const size_t smem = (size_t)RG * sap_group_smem<R>(g.Vb / 2);
  set_dynamic_smem((const void*)k_sap_half<P, RG>, smem);
  // grid.y is at most 65535: on large lattices (e.g. 128 x 64^3 with 4^4 blocks, 65536 blocks per
  // colour) the blocks of the colour go in several launches, which is exact since they are independent
  for (int b0 = 0; b0 < nblocks; b0 += 65535) {
    const int nb = nblocks - b0 < 65535 ? nblocks - b0 : 65535;
    SapArgs<R> a{blocks + b0, nrhs, zero_blocks + b0, zero_x, nmr, (R)mu, (size_t)g.V * 12, g.V};
    dim3 grid((nrhs + RG - 1) / RG, nb);
    k_sap_half<P, RG><<<grid, RG * sap_threads(g.Vb), smem, s>>>(
        Spinor<P>{(S*)x, xn, g.Vb}, Spinor<P>{(S*)b, (float*)bn, g.Vb}, Links<P>{(const S*)links, g.Vb},
        Clover<P>{(const S*)clover, g.Vb}, SiteInv<P>{(const S*)sinv, g.Vb / 2}, q, a);
    CKL("sap_half");
  }
}

// Right-hand sides per CTA: up to DDTM_SAP_RG where the batch and the shared memory allow it, fewer
// otherwise; FP64 keeps one.  Two per CTA (99 KB of FP32 block vectors for 4^4 blocks, 2 CTAs per
// SM) measured fastest at 32^3 x 64 with 12 and 24 right-hand sides: 34.7 / 68.9 ms per two cycles,
// against 36.7 / 74.2 ms with one and 37.3 / 73.8 ms with four (whose 198 KB of shared memory leave
// little L1 for the shared operator data).
#ifndef DDTM_SAP_RG
#define DDTM_SAP_RG 2
#endif
static int sap_rhs_groups(const FineGeom& g, int prec, int nrhs) {
  if (prec == PREC_F64 || nrhs <= 1) return 1;
  const size_t grp = sap_group_smem<float>(g.Vb / 2);
  const int gt = sap_threads(g.Vb);
  if (DDTM_SAP_RG >= 4 && nrhs >= 3 && 4 * grp <= 200 * 1024 && 4 * gt <= 1024) return 4;
  if (DDTM_SAP_RG >= 2 && 2 * grp <= 200 * 1024 && 2 * gt <= 1024) return 2;
  return 1;
}

template <int P>
static void launch_sap_half_t(const FineGeom& g, void* x, float* xn, const void* b, const float* bn, const void* links,
                              const void* clover, const void* sinv, const int* blocks, const int* zero_blocks,
                              int nblocks, int zero_x, int nmr, double mu, int nrhs, cudaStream_t s) {
  const int rg = sap_rhs_groups(g, P, nrhs);
  if constexpr (P != PREC_F64) {
    if (rg == 4) {
      launch_sap_rg<P, 4>(g, x, xn, b, bn, links, clover, sinv, blocks, zero_blocks, nblocks, zero_x, nmr, mu, nrhs, s);
      return;
    }
    if (rg == 2) {
      launch_sap_rg<P, 2>(g, x, xn, b, bn, links, clover, sinv, blocks, zero_blocks, nblocks, zero_x, nmr, mu, nrhs, s);
      return;
    }
  }
  launch_sap_rg<P, 1>(g, x, xn, b, bn, links, clover, sinv, blocks, zero_blocks, nblocks, zero_x, nmr, mu, nrhs, s);
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

// Per-site pieces of D(mu) (Sec. 2.1) used by several kernels: the full
// stencil at one site, and the hop restricted to one lattice block with
// Dirichlet block boundaries (Sec. 2.4) acting on a block vector held in
// shared memory.
#pragma once

#include "common.cuh"

namespace ddtm {

// out = D(mu) x at internal site (blk, loc): clover + twist + 8 hops.
// UNROLL = 1 keeps the direction loop rolled (register pressure inside SAP).
template <int P, int UNROLL = 4>
__device__ __forceinline__ void dslash_site(const Spinor<P>& x, const Links<P>& U, const Clover<P>& C, const Geo& g,
                                            typename Prec<P>::real mu, int blk, int loc,
                                            cplx<typename Prec<P>::real> out[12]) {
  typedef typename Prec<P>::real R;
  cplx<R> acc[12];
#pragma unroll
  for (int c = 0; c < 12; c++) acc[c] = cplx<R>(0, 0);
#pragma unroll (UNROLL)
  for (int mu_ = 0; mu_ < 4; mu_++) {
#pragma unroll (UNROLL == 1 ? 1 : 2)
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
  cplx<R> in[12];
  x.load(blk, loc, in);
  C.apply(blk, loc, in, out);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    R m = c < 6 ? mu : -mu;
    out[c] = out[c] + m * times_i(in[c]) + R(-0.5) * acc[c];
  }
}

// Block vector in shared memory: v[c * Vh + i] holds component c of the site
// with parity-local index i (loc = parity * Vh + i).
// out = H_B v at site loc: the hopping term of D restricted to the block
// (hops leaving the block are dropped), reading v on the sites of the other
// parity.  Links are read from global memory.
template <int P, typename R>
__device__ __forceinline__ void hop_block(const cplx<R>* v, int Vh, const Links<P>& U, const Geo& g, int blk, int loc,
                                          cplx<R> out[12]) {
  cplx<R> acc[12];
#pragma unroll
  for (int c = 0; c < 12; c++) acc[c] = cplx<R>(0, 0);
#pragma unroll 1
  for (int mu_ = 0; mu_ < 4; mu_++) {
#pragma unroll 1
    for (int dir = 0; dir < 2; dir++) {
      bool fwd = dir == 0;
      uint32_t e = __ldg(g.loc_nbr + (2 * mu_ + dir) * g.Vb + loc);
      if ((e >> 16) & 1) continue;  // Dirichlet: the hop leaves the block
      int nloc = e & 0xffff;
      int ni = nloc >= Vh ? nloc - Vh : nloc;
      cplx<R> h[6], w[6], u[9];
      {
        cplx<R> p[12];
#pragma unroll
        for (int c = 0; c < 12; c++) p[c] = v[c * Vh + ni];
        project<R>(mu_, fwd, p, h);
      }
      if (fwd) {
        U.load(blk, loc, mu_, u);
        mul_U<R>(u, h, w);
      } else {
        U.load(blk, nloc, mu_, u);
        mul_Udag<R>(u, h, w);
      }
      reconstruct<R>(mu_, fwd, w, acc);
    }
  }
#pragma unroll
  for (int c = 0; c < 12; c++) out[c] = R(-0.5) * acc[c];
}

}  // namespace ddtm

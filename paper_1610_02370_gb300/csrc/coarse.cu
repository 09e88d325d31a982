// Coarse operator D_c(mu) = P^dagger D P + i mu Gamma5_c (Sec. 2.3): Galerkin
// build, stencil, even-odd reduction pieces, and the self-block inverses of
// the even-odd coarsest solve (Sec. 2.5).
//
// Storage: Dc[((x*9 + d)*n + col)*n + row], complex FP32, n = 2 nv,
// d = 0 self (without the twist), d = 1 + k for hop k = 2 mu + (0 fwd, 1 bwd):
// the block coupling site x to its neighbour in direction +mu (k even) or
// -mu (k odd).  Column-major blocks make the per-row threads of the stencil
// read consecutive addresses.  The twist i mu_c Gamma5_c (Gamma5_c = +1 on
// dofs < nv, -1 above) is added on the fly, so one build serves +mu, -mu and
// the shifted coarsest twist delta*mu.  With FP16 coarse storage the stencil
// of the coarsest solve runs on tensor cores from FP16 images of these blocks
// (coarse_tc.cu); the FP32 blocks stay for the rest.
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"
#include "coarse.h"
#include "launch_shape.h"

namespace ddtm {

template <typename DS> __device__ __forceinline__ cplx<float> ldD(const DS* p);
template <> __device__ __forceinline__ cplx<float> ldD<float2>(const float2* p) { return ld(p); }
template <typename DS> __device__ __forceinline__ void stD(DS* p, cplx<float> v);
template <> __device__ __forceinline__ void stD<float2>(float2* p, cplx<float> v) { st(p, v); }

__device__ __forceinline__ size_t pix(int blk, int s, int i, int comp, int loc, int nv, int Vb) {
  return (((size_t)(blk * 2 + s) * nv + i) * 6 + comp) * Vb + loc;
}

// ---- Galerkin build ----------------------------------------------------------------
// One CTA per aggregate A, thread = site.  For every column (s', j) of P:
//   y0(x)  = S phi(x) + hops of phi that stay inside A          (self part)
//   yk(x)  = hop k of phi read in the neighbour aggregate, for x on face k
// with phi = column (s', j) of every aggregate; then
//   Dc[A][0][col][row]   = sum_{x in A} <P_row(x), y0(x)>
//   Dc[A][1+k][col][row] = sum_{x on face k} <P_row(x), yk(x)>
// Face k of a block = sites whose hop k leaves the block; faces are stored
// compactly (face_list / face_idx tables, offsets face_off).
struct FaceTables {
  const int* idx;   // [8][Vb]: slot of site in face k or -1
  const int* list;  // [face_off[8]]: site of each slot
  int off[9];
};

template <typename DS>
__global__ void k_galerkin(DS* __restrict__ Dc, const float2* __restrict__ P, Links<PREC_F32> U, Clover<PREC_F32> C,
                           Geo g, FaceTables f, int nv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vb = g.Vb;
  cplx<float>* y0 = reinterpret_cast<cplx<float>*>(smem_raw);  // [12][Vb]
  cplx<float>* yf = y0 + 12 * Vb;                                // [12][face slots]
  const int nf = f.off[8];
  const int A = blockIdx.x;
  const int n = 2 * nv;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int col = 0; col < n; col++) {
    const int sp = col / nv, j = col - sp * nv;
    for (int loc = threadIdx.x; loc < Vb; loc += blockDim.x) {
      cplx<float> phi[12], acc[12], out[12];
#pragma unroll
      for (int c = 0; c < 12; c++) { phi[c] = cplx<float>(0, 0); acc[c] = cplx<float>(0, 0); }
      for (int comp = 0; comp < 6; comp++) phi[6 * sp + comp] = ld(P + pix(A, sp, j, comp, loc, nv, Vb));
      C.apply(A, loc, phi, out);
      for (int k = 0; k < 8; k++) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        Nbr nb = neighbour(g, A, loc, k);
        cplx<float> p[12], h[6], wv[6], u[9];
#pragma unroll
        for (int c = 0; c < 12; c++) p[c] = cplx<float>(0, 0);
        for (int comp = 0; comp < 6; comp++) p[6 * sp + comp] = ld(P + pix(nb.blk, sp, j, comp, nb.loc, nv, Vb));
        project<float>(mu, fwd, p, h);
        if (fwd) { U.load(A, loc, mu, u); mul_U<float>(u, h, wv); }
        else { U.load(nb.blk, nb.loc, mu, u); mul_Udag<float>(u, h, wv); }
        if (nb.flip)
          for (int q = 0; q < 6; q++) wv[q] = -wv[q];
        if (!nb.cross) {
          reconstruct<float>(mu, fwd, wv, acc);
        } else {
          cplx<float> part[12];
#pragma unroll
          for (int c = 0; c < 12; c++) part[c] = cplx<float>(0, 0);
          reconstruct<float>(mu, fwd, wv, part);
          int slot = f.off[k] + f.idx[k * Vb + loc];
#pragma unroll
          for (int c = 0; c < 12; c++) yf[c * nf + slot] = -0.5f * part[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 12; c++) y0[c * Vb + loc] = out[c] + (-0.5f) * acc[c];
    }
    __syncthreads();
    // projections: a warp takes GR rows of one block d (independent loads of
    // GR rows of P per step), the lanes stride over the sites
    const int GR = 4, ngr = (n + GR - 1) / GR;
    for (int o = w; o < 9 * ngr; o += nw) {
      const int d = o / ngr, r0 = (o - d * ngr) * GR;
      cplx<float> acc[GR];
      int sr[GR], ir[GR];
#pragma unroll
      for (int r = 0; r < GR; r++) {
        acc[r] = cplx<float>(0, 0);
        const int row = r0 + r < n ? r0 + r : n - 1;
        sr[r] = row / nv;
        ir[r] = row - sr[r] * nv;
      }
      if (d == 0) {
        for (int comp = 0; comp < 6; comp++)
#pragma unroll 4
          for (int loc = lane; loc < Vb; loc += 32)
#pragma unroll
            for (int r = 0; r < GR; r++)
              cmac_conj(acc[r], ld(P + pix(A, sr[r], ir[r], comp, loc, nv, Vb)), y0[(6 * sr[r] + comp) * Vb + loc]);
      } else {
        const int k = d - 1;
        for (int comp = 0; comp < 6; comp++)
#pragma unroll 2
          for (int q = f.off[k] + lane; q < f.off[k + 1]; q += 32) {
            const int fl = f.list[q];
#pragma unroll
            for (int r = 0; r < GR; r++)
              cmac_conj(acc[r], ld(P + pix(A, sr[r], ir[r], comp, fl, nv, Vb)), yf[(6 * sr[r] + comp) * nf + q]);
          }
      }
#pragma unroll
      for (int r = 0; r < GR; r++) {
        acc[r].re = warp_sum(acc[r].re);
        acc[r].im = warp_sum(acc[r].im);
        if (lane == 0 && r0 + r < n) stD(Dc + (((size_t)A * 9 + d) * n + col) * n + r0 + r, acc[r]);
      }
    }
    __syncthreads();
  }
}

// The same Galerkin products with the rows staged in shared memory, for FP16
// coarse storage (the tensor-core images round D_c to FP16 anyway): one CTA
// per (aggregate A, row chirality s) keeps the nv rows (s, i) of P on A as
// FP16 in shared memory, computes for CC columns (s', j) at a time the
// chirality-s components of y_0 and of the face hops y_k as above (each link
// loaded once for the CC columns), and projects them out of shared memory, each
// row entry loaded once for the CC columns, so P is not re-read from memory
// for every column and the projections need fewer shared-memory loads per
// multiply-add.  Every entry is the same sum, in the same order, for any CC.
template <int CC>
__global__ void __launch_bounds__(256, 1) k_galerkin_rows(float2* __restrict__ Dc, const float2* __restrict__ P,
                                                          Links<PREC_F32> U, Clover<PREC_F32> C, Geo g, FaceTables f,
                                                          int nv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vb = g.Vb, nf = f.off[8];
  const int A = blockIdx.x >> 1, s = blockIdx.x & 1;
  const int n = 2 * nv;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __half2* Ps = reinterpret_cast<__half2*>(smem_raw);                                // [nv][6][Vb]
  cplx<float>* y0 = reinterpret_cast<cplx<float>*>(Ps + (size_t)nv * 6 * Vb);          // [CC][6][Vb]
  cplx<float>* yf = y0 + (size_t)CC * 6 * Vb;                                          // [CC][6][nf]
  const size_t rows0 = pix(A, s, 0, 0, 0, nv, Vb);
  for (int e = threadIdx.x; e < nv * 6 * Vb; e += blockDim.x) Ps[e] = __float22half2_rn(__ldg(P + rows0 + e));
  for (int col0 = 0; col0 < n; col0 += CC) {
    const int ncol = n - col0 < CC ? n - col0 : CC;
    for (int loc = threadIdx.x; loc < Vb; loc += blockDim.x) {
      cplx<float> acc[CC][12];
#pragma unroll
      for (int cc = 0; cc < CC; cc++)
#pragma unroll
        for (int c = 0; c < 12; c++) acc[cc][c] = cplx<float>(0, 0);
      for (int k = 0; k < 8; k++) {
        const int mu = k >> 1;
        const bool fwd = (k & 1) == 0;
        Nbr nb = neighbour(g, A, loc, k);
        cplx<float> u[9];
        if (fwd) U.load(A, loc, mu, u);
        else U.load(nb.blk, nb.loc, mu, u);
        const int slot = nb.cross ? f.off[k] + f.idx[k * Vb + loc] : 0;
#pragma unroll
        for (int cc = 0; cc < CC; cc++) {
          if (cc >= ncol) break;
          const int col = col0 + cc, sp = col / nv, j = col - sp * nv;
          cplx<float> p[12], h[6], wv[6];
#pragma unroll
          for (int c = 0; c < 12; c++)  // column (sp, j): chirality-sp components only (static indices)
            p[c] = (c / 6 == sp) ? ld(P + pix(nb.blk, sp, j, c % 6, nb.loc, nv, Vb)) : cplx<float>(0, 0);
          project<float>(mu, fwd, p, h);
          if (fwd) mul_U<float>(u, h, wv);
          else mul_Udag<float>(u, h, wv);
          if (nb.flip)
            for (int q = 0; q < 6; q++) wv[q] = -wv[q];
          if (!nb.cross) {
            reconstruct<float>(mu, fwd, wv, acc[cc]);
          } else {
            cplx<float> part[12];
#pragma unroll
            for (int c = 0; c < 12; c++) part[c] = cplx<float>(0, 0);
            reconstruct<float>(mu, fwd, wv, part);
#pragma unroll
            for (int c = 0; c < 6; c++) yf[((size_t)cc * 6 + c) * nf + slot] = -0.5f * (s ? part[6 + c] : part[c]);
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < CC; cc++) {
        if (cc >= ncol) break;
        const int col = col0 + cc, sp = col / nv, j = col - sp * nv;
        cplx<float> phi[12], out[12];
#pragma unroll
        for (int c = 0; c < 12; c++)
          phi[c] = (c / 6 == sp) ? ld(P + pix(A, sp, j, c % 6, loc, nv, Vb)) : cplx<float>(0, 0);
        C.apply(A, loc, phi, out);
#pragma unroll
        for (int c = 0; c < 6; c++)
          y0[((size_t)cc * 6 + c) * Vb + loc] = s ? out[6 + c] + (-0.5f) * acc[cc][6 + c] : out[c] + (-0.5f) * acc[cc][c];
      }
    }
    __syncthreads();
    const int GR = 4, ngr = (nv + GR - 1) / GR;
    for (int o = w; o < 9 * ngr; o += nw) {
      const int d = o / ngr, r0 = (o - d * ngr) * GR;
      cplx<float> acc[GR][CC];
      int ir[GR];
#pragma unroll
      for (int r = 0; r < GR; r++) {
#pragma unroll
        for (int cc = 0; cc < CC; cc++) acc[r][cc] = cplx<float>(0, 0);
        ir[r] = r0 + r < nv ? r0 + r : nv - 1;
      }
      if (d == 0) {
        for (int comp = 0; comp < 6; comp++)
#pragma unroll 4
          for (int loc = lane; loc < Vb; loc += 32) {
            cplx<float> yv[CC];
#pragma unroll
            for (int cc = 0; cc < CC; cc++) yv[cc] = y0[((size_t)cc * 6 + comp) * Vb + loc];
#pragma unroll
            for (int r = 0; r < GR; r++) {
              const float2 pv = __half22float2(Ps[((size_t)ir[r] * 6 + comp) * Vb + loc]);
#pragma unroll
              for (int cc = 0; cc < CC; cc++) cmac_conj(acc[r][cc], cplx<float>(pv.x, pv.y), yv[cc]);
            }
          }
      } else {
        const int k = d - 1;
        for (int comp = 0; comp < 6; comp++)
#pragma unroll 2
          for (int q = f.off[k] + lane; q < f.off[k + 1]; q += 32) {
            const int fl = f.list[q];
            cplx<float> yv[CC];
#pragma unroll
            for (int cc = 0; cc < CC; cc++) yv[cc] = yf[((size_t)cc * 6 + comp) * nf + q];
#pragma unroll
            for (int r = 0; r < GR; r++) {
              const float2 pv = __half22float2(Ps[((size_t)ir[r] * 6 + comp) * Vb + fl]);
#pragma unroll
              for (int cc = 0; cc < CC; cc++) cmac_conj(acc[r][cc], cplx<float>(pv.x, pv.y), yv[cc]);
            }
          }
      }
#pragma unroll
      for (int r = 0; r < GR; r++)
#pragma unroll
        for (int cc = 0; cc < CC; cc++) {
          acc[r][cc].re = warp_sum(acc[r][cc].re);
          acc[r][cc].im = warp_sum(acc[r][cc].im);
          if (lane == 0 && r0 + r < nv && cc < ncol)
            Dc[(((size_t)A * 9 + d) * n + col0 + cc) * n + s * nv + r0 + r] = make_float2(acc[r][cc].re, acc[r][cc].im);
        }
    }
    __syncthreads();
  }
}

static size_t galerkin_rows_smem(const FineGeom& g, const FaceDev& faces, int nv, int cc) {
  return (size_t)nv * 6 * g.Vb * sizeof(__half2) + (size_t)cc * 6 * (g.Vb + faces.off[8]) * sizeof(cplx<float>);
}

void launch_galerkin(const FineGeom& g, const FaceDev& faces, int dprec, void* Dc, const float2* P, const void* links32,
                     const void* clover32, int nv, bool rows_fp16, cudaStream_t st) {
  ScopedTimer timer_("galerkin", st);
  Geo q{g.Vb, g.Nb, g.loc_nbr.as<uint32_t>(), g.blk_nbr.as<int>()};
  FaceTables f;
  f.idx = faces.idx.as<int>();
  f.list = faces.list.as<int>();
  for (int k = 0; k < 9; k++) f.off[k] = faces.off[k];
  size_t smem = (size_t)12 * (g.Vb + faces.off[8]) * sizeof(cplx<float>);
  int threads = g.Vb >= 256 ? 256 : ((g.Vb + 31) / 32) * 32;
  Links<PREC_F32> U{(const float2*)links32, g.Vb};
  Clover<PREC_F32> C{(const float2*)clover32, g.Vb};
  if (dprec != PREC_F32) throw Error(DDTM_ERR_ARG, "internal: Galerkin output is FP32");
  const size_t srows1 = galerkin_rows_smem(g, faces, nv, 1), srows2 = galerkin_rows_smem(g, faces, nv, 2);
  if (rows_fp16 && srows2 <= 224 * 1024) {  // two columns per pass where the shared memory holds them
    set_dynamic_smem((const void*)k_galerkin_rows<2>, srows2);
    k_galerkin_rows<2><<<g.Nb * 2, threads, srows2, st>>>((float2*)Dc, P, U, C, q, f, nv);
  } else if (rows_fp16 && srows1 <= 220 * 1024) {
    set_dynamic_smem((const void*)k_galerkin_rows<1>, srows1);
    k_galerkin_rows<1><<<g.Nb * 2, threads, srows1, st>>>((float2*)Dc, P, U, C, q, f, nv);
  } else {
    set_dynamic_smem((const void*)k_galerkin<float2>, smem);
    k_galerkin<float2><<<g.Nb, threads, smem, st>>>((float2*)Dc, P, U, C, q, f, nv);
  }
  CKL("galerkin");
}

void build_faces(const FineGeom& g, FaceDev& faces) {
  std::vector<int> idx(8 * g.Vb, -1), list;
  for (int k = 0; k < 8; k++) {
    faces.off[k] = (int)list.size();
    for (int loc = 0; loc < g.Vb; loc++)
      if ((g.h_loc_nbr[k * g.Vb + loc] >> 16) & 1) {
        idx[k * g.Vb + loc] = (int)list.size() - faces.off[k];
        list.push_back(loc);
      }
  }
  faces.off[8] = (int)list.size();
  faces.idx.ensure(idx.size() * 4);
  faces.list.ensure(list.size() * 4 + 4);
  CK(cudaMemcpy(faces.idx.p, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(faces.list.p, list.data(), list.size() * 4, cudaMemcpyHostToDevice));
}

// ---- coarse stencil ---------------------------------------------------------------
// Coarse vectors of a batch of R right-hand sides are stored interleaved,
// v[(idx * n + k) * R + r], so the R values of one dof are contiguous.  A
// thread owns one row r of one site and RC consecutive right-hand sides
// (register blocking: each matrix entry read from HBM is used RC times by the
// thread and R / RC times by the site's threads); threads of a site are
// ordered row fastest, so a warp reads consecutive entries of a column-major
// block.  Output slot idx has lattice site osite[idx] (idx itself when
// osite == nullptr); the self term reads x_self[idx], hop d reads
// x_hop[tab[(d-1) * nout + idx]] (tab: full neighbour table for full-lattice
// vectors, or the parity-compact table into the other parity's vector).
//   mode & 1: self block + twist i mu_c Gamma5_c;  mode & 2: the 8 hops
//   y[idx] = sy * y[idx] + sres * result   (sy = 0 overwrites y)
template <int RC>
__device__ __forceinline__ void load_rc(const cplx<float>* p, cplx<float> v[RC]) {
  if (RC == 4) {
    const float4* q = reinterpret_cast<const float4*>(p);
    float4 a = q[0], b = q[1];
    v[0] = cplx<float>(a.x, a.y); v[1] = cplx<float>(a.z, a.w);
    v[2] = cplx<float>(b.x, b.y); v[3] = cplx<float>(b.z, b.w);
  } else if (RC == 2) {
    float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = cplx<float>(a.x, a.y); v[1] = cplx<float>(a.z, a.w);
  } else {
#pragma unroll
    for (int c = 0; c < RC; c++) v[c] = p[c];
  }
}

// Two consecutive rows (r, r+1) of column k of a column-major block: one
// 16-byte load.
template <typename DS> __device__ __forceinline__ void ld_rows2(const DS* p, cplx<float>& a0, cplx<float>& a1);
template <> __device__ __forceinline__ void ld_rows2<float2>(const float2* p, cplx<float>& a0, cplx<float>& a1) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a0 = cplx<float>(v.x, v.y);
  a1 = cplx<float>(v.z, v.w);
}

// acc{0,1}[c] += A[r0 + {0,1}][k] v[k][c] for a column-major n x n block whose
// row r0 is at A; the column loop is unrolled so that many independent
// matrix loads are in flight per thread.
template <typename DS, int RC>
__device__ __forceinline__ void block_mv2(const DS* A, const cplx<float>* v, int n, int R, cplx<float> acc0[RC],
                                          cplx<float> acc1[RC]) {
#pragma unroll 8
  for (int k = 0; k < n; k++) {
    cplx<float> a0, a1;
    ld_rows2<DS>(A + (size_t)k * n, a0, a1);
    cplx<float> x[RC];
    load_rc<RC>(v + (size_t)k * R, x);
#pragma unroll
    for (int c = 0; c < RC; c++) {
      cmac(acc0[c], a0, x[c]);
      cmac(acc1[c], a1, x[c]);
    }
  }
}

// Threads of a site: n/2 row pairs x G chunk slots, row pair fastest (a warp
// reads consecutive 16-byte pieces of a column); a thread takes the chunks
// ch = g, g + G, ... of RC right-hand sides (launch_shape.h); SPB sites per CTA.
template <typename DS, int RC>
__global__ void __launch_bounds__(256) k_coarse_apply(cplx<float>* __restrict__ y, const cplx<float>* __restrict__ x_self,
                                                       const cplx<float>* __restrict__ x_hop, const DS* __restrict__ Dc,
                                                       const int* __restrict__ tab, const int* __restrict__ osite, int nout,
                                                       int n, int nv, int R, int G, float mu_c, int mode, float sres,
                                                       float sy, int dsel) {
  const int np = n / 2, nch = R / RC, per = np * G, spb = blockDim.x / per;
  const int t = threadIdx.x, rp = t % np, g = (t / np) % G, q = t / per;
  const int idx = blockIdx.x * spb + q;
  if (q >= spb || idx >= nout) return;
  const int site = osite ? osite[idx] : idx;
  const int r0 = 2 * rp;
  for (int ch = g; ch < nch; ch += G) {
  const int c0 = ch * RC;
  cplx<float> acc0[RC], acc1[RC];
#pragma unroll
  for (int c = 0; c < RC; c++) acc0[c] = acc1[c] = cplx<float>(0, 0);
  if (mode & 1) {
    block_mv2<DS, RC>(Dc + (size_t)site * 9 * n * n + r0, x_self + (size_t)idx * n * R + c0, n, R, acc0, acc1);
    cplx<float> xv0[RC], xv1[RC];
    load_rc<RC>(x_self + ((size_t)idx * n + r0) * R + c0, xv0);
    load_rc<RC>(x_self + ((size_t)idx * n + r0 + 1) * R + c0, xv1);
    const float m0 = r0 < nv ? mu_c : -mu_c, m1 = r0 + 1 < nv ? mu_c : -mu_c;
#pragma unroll
    for (int c = 0; c < RC; c++) {
      acc0[c] = acc0[c] + m0 * times_i(xv0[c]);
      acc1[c] = acc1[c] + m1 * times_i(xv1[c]);
    }
  }
  if (mode & 2)
    for (int d = dsel ? dsel : 1; d <= (dsel ? dsel : 8); d++) {  // dsel > 0: hop dsel - 1 only
      const int src = __ldg(tab + (size_t)(d - 1) * nout + idx);
      block_mv2<DS, RC>(Dc + ((size_t)site * 9 + d) * n * n + r0, x_hop + (size_t)src * n * R + c0, n, R, acc0, acc1);
    }
  cplx<float>* yo0 = y + ((size_t)idx * n + r0) * R + c0;
  cplx<float>* yo1 = yo0 + R;
#pragma unroll
  for (int c = 0; c < RC; c++) {
    cplx<float> res0 = sres * acc0[c], res1 = sres * acc1[c];
    yo0[c] = sy == 0.f ? res0 : sy * yo0[c] + res0;
    yo1[c] = sy == 0.f ? res1 : sy * yo1[c] + res1;
  }
  }
}

// t[e] = Dinv_e (sr * rhs[e] + sh * hops(v)) on the even sites (compact even
// output, v compact odd); rhs or v may be null.  Hop and inverse are fused:
// the hop result of a site goes through shared memory to the threads of the
// same site for the dense matvec with the inverse.
template <typename DS, int RC>
__global__ void __launch_bounds__(256) k_coarse_even(cplx<float>* __restrict__ t, const cplx<float>* __restrict__ rhs,
                                                      const cplx<float>* __restrict__ v, const DS* __restrict__ Dc,
                                                      const float2* __restrict__ Dinv, const int* __restrict__ tab,
                                                      const int* __restrict__ even, int ne, int n, int R, int G, float sr,
                                                      float sh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int np = n / 2, nch = R / RC, per = np * G, spb = blockDim.x / per;
  cplx<float>* hs = reinterpret_cast<cplx<float>*>(smem_raw);  // [spb][n][R]
  const int th = threadIdx.x, rp = th % np, g = (th / np) % G, q = th / per;
  const int e = blockIdx.x * spb + q;
  const bool act = q < spb && e < ne;
  const int r0 = 2 * rp;
  if (act)
  for (int ch = g; ch < nch; ch += G) {
    const int c0 = ch * RC;
    const int site = even[e];
    cplx<float> acc0[RC], acc1[RC];
#pragma unroll
    for (int c = 0; c < RC; c++) acc0[c] = acc1[c] = cplx<float>(0, 0);
    if (v)
      for (int d = 1; d < 9; d++) {
        const int src = __ldg(tab + (size_t)(d - 1) * ne + e);
        block_mv2<DS, RC>(Dc + ((size_t)site * 9 + d) * n * n + r0, v + (size_t)src * n * R + c0, n, R, acc0, acc1);
      }
    cplx<float> rv0[RC], rv1[RC];
    if (rhs) {
      load_rc<RC>(rhs + ((size_t)e * n + r0) * R + c0, rv0);
      load_rc<RC>(rhs + ((size_t)e * n + r0 + 1) * R + c0, rv1);
    }
#pragma unroll
    for (int c = 0; c < RC; c++) {
      cplx<float> a0 = sh * acc0[c], a1 = sh * acc1[c];
      if (rhs) {
        a0 = a0 + sr * rv0[c];
        a1 = a1 + sr * rv1[c];
      }
      hs[((size_t)q * n + r0) * R + c0 + c] = a0;
      hs[((size_t)q * n + r0 + 1) * R + c0 + c] = a1;
    }
  }
  __syncthreads();
  if (act)
  for (int ch = g; ch < nch; ch += G) {
    const int c0 = ch * RC;
    cplx<float> o0[RC], o1[RC];
#pragma unroll
    for (int c = 0; c < RC; c++) o0[c] = o1[c] = cplx<float>(0, 0);
    block_mv2<float2, RC>(Dinv + (size_t)e * n * n + r0, hs + (size_t)q * n * R + c0, n, R, o0, o1);
    cplx<float>* to0 = t + ((size_t)e * n + r0) * R + c0;
    cplx<float>* to1 = to0 + R;
#pragma unroll
    for (int c = 0; c < RC; c++) {
      to0[c] = o0[c];
      to1[c] = o1[c];
    }
  }
}

// gather (dir = 0: compact[i] = full[list[i]]) or scatter (dir = 1), n*R
// contiguous complex numbers per site
__global__ void k_parity_copy(cplx<float>* __restrict__ compact, cplx<float>* __restrict__ full, const int* __restrict__ list,
                              int cnt, int nr, int dir) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)cnt * nr) return;
  int i = (int)(t / nr), r = (int)(t - (size_t)i * nr);
  size_t f = (size_t)list[i] * nr + r;
  if (dir == 0) compact[t] = full[f];
  else full[f] = compact[t];
}

// canonical FP64 coarse vector c[site * n + k] <-> column r of an interleaved
// FP32 batch v[(site * n + k) * R + r] (dir 0: c -> v, dir 1: v -> c)
__global__ void k_coarse_interleave(float2* __restrict__ v, double* __restrict__ c, size_t nc, int r, int R, int dir) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  if (dir == 0) {
    v[t * R + r] = make_float2((float)c[2 * t], (float)c[2 * t + 1]);
  } else {
    float2 z = v[t * R + r];
    c[2 * t] = z.x;
    c[2 * t + 1] = z.y;
  }
}

// Inverse of (self block + i mu_c Gamma5_c) per even site by Gauss-Jordan
// elimination with partial pivoting in CT (FP64, or FP32 where the inverses
// only feed FP16 operator images); one CTA per site, thread = row.
template <typename DS, typename CT>
__global__ void k_self_inverse(float2* __restrict__ Dinv, const DS* __restrict__ Dc, const int* __restrict__ even, int n,
                               int nv, double mu_c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<CT>* M = reinterpret_cast<cplx<CT>*>(smem_raw);  // [n][2n] row-major augmented
  __shared__ int piv;
  const int e = blockIdx.x, site = even[e];
  const int r = threadIdx.x;
  const int w2 = 2 * n;
  if (r < n) {
    for (int c = 0; c < n; c++) {
      cplx<float> a = ldD<DS>(Dc + ((size_t)site * 9 * n + c) * n + r);  // d = 0, column c, row r
      M[r * w2 + c] = cplx<CT>((CT)a.re, (CT)a.im);
      M[r * w2 + n + c] = cplx<CT>(r == c ? CT(1) : CT(0), CT(0));
    }
    M[r * w2 + r].im += (CT)(r < nv ? mu_c : -mu_c);
  }
  __syncthreads();
  for (int c = 0; c < n; c++) {
    if (r == 0) {
      int p = c;
      CT best = norm2(M[c * w2 + c]);
      for (int k = c + 1; k < n; k++)
        if (norm2(M[k * w2 + c]) > best) { best = norm2(M[k * w2 + c]); p = k; }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != c && r < w2) {  // swap rows c and p, column r (and r + n) per thread
      for (int cc = r; cc < w2; cc += blockDim.x) {
        cplx<CT> tmp = M[c * w2 + cc];
        M[c * w2 + cc] = M[p * w2 + cc];
        M[p * w2 + cc] = tmp;
      }
    }
    __syncthreads();
    cplx<CT> d = M[c * w2 + c];
    CT dn = norm2(d);
    cplx<CT> inv(d.re / dn, -d.im / dn);
    __syncthreads();
    for (int cc = r; cc < w2; cc += blockDim.x) M[c * w2 + cc] = M[c * w2 + cc] * inv;
    __syncthreads();
    if (r < n && r != c) {
      cplx<CT> fct = M[r * w2 + c];
      for (int cc = 0; cc < w2; cc++) M[r * w2 + cc] = M[r * w2 + cc] - fct * M[c * w2 + cc];
    }
    __syncthreads();
  }
  if (r < n)
    for (int c = 0; c < n; c++) {
      cplx<CT> v = M[r * w2 + n + c];
      Dinv[((size_t)e * n + c) * n + r] = make_float2((float)v.re, (float)v.im);  // column-major
    }
}

template <typename DS, int RC>
static void coarse_apply_t(const CoarseLevel& c, const CoarseShape& sh, cplx<float>* y, const cplx<float>* xs,
                           const cplx<float>* xh, const int* tab, const int* osite, int nout, int R, double mu_c, int mode,
                           float sres, float sy, cudaStream_t st, int dsel) {
  unsigned grid = (unsigned)((nout + sh.spb - 1) / sh.spb);
  if (grid == 0) return;
  k_coarse_apply<DS, RC><<<grid, sh.threads, 0, st>>>(y, xs, xh, c.Dc.as<DS>(), tab, osite, nout, c.n, c.nv, R, sh.groups,
                                                      (float)mu_c, mode, sres, sy, dsel);
  CKL("coarse_apply");
}

template <typename DS>
static void coarse_apply_d(const CoarseLevel& c, cplx<float>* y, const cplx<float>* xs, const cplx<float>* xh, const int* tab,
                           const int* osite, int nout, int R, double mu_c, int mode, float sres, float sy, cudaStream_t st,
                           int dsel = 0) {
  const CoarseShape sh = coarse_shape(c.n, R);
  if (sh.rc == 4) coarse_apply_t<DS, 4>(c, sh, y, xs, xh, tab, osite, nout, R, mu_c, mode, sres, sy, st, dsel);
  else if (sh.rc == 2) coarse_apply_t<DS, 2>(c, sh, y, xs, xh, tab, osite, nout, R, mu_c, mode, sres, sy, st, dsel);
  else coarse_apply_t<DS, 1>(c, sh, y, xs, xh, tab, osite, nout, R, mu_c, mode, sres, sy, st, dsel);
}

void launch_coarse_apply_hop(const CoarseLevel& c, cplx<float>* y, const cplx<float>* x, int R, int hop, cudaStream_t st) {
  ScopedTimer timer_("coarse_apply", st, R);
  coarse_apply_d<float2>(c, y, x, x, c.nbr.as<int>(), nullptr, c.Nc, R, 0.0, 2, 1.f, 0.f, st, hop + 1);
}

void launch_coarse_apply_full(const CoarseLevel& c, cplx<float>* y, const cplx<float>* x, int R, double mu_c, int mode,
                              float sres, float sy, cudaStream_t st) {
  ScopedTimer timer_("coarse_apply", st, R);
  coarse_apply_d<float2>(c, y, x, x, c.nbr.as<int>(), nullptr, c.Nc, R, mu_c, mode, sres, sy, st);
}

void launch_coarse_apply_odd(const CoarseLevel& c, cplx<float>* y_o, const cplx<float>* x_o, const cplx<float>* x_e, int R,
                             double mu_c, int mode, float sres, float sy, cudaStream_t st) {
  ScopedTimer timer_("coarse_apply_odd_f32", st, R);
  int no = (int)c.h_odd.size();
  coarse_apply_d<float2>(c, y_o, x_o, x_e, c.nbr_oe.as<int>(), c.odd.as<int>(), no, R, mu_c, mode, sres, sy, st);
}

template <typename DS, int RC>
static void coarse_even_t(const CoarseLevel& c, const CoarseShape& shp, cplx<float>* t, const cplx<float>* rhs,
                          const cplx<float>* v, int R, float sr, float sh, cudaStream_t st) {
  int ne = (int)c.h_even.size();
  unsigned grid = (unsigned)((ne + shp.spb - 1) / shp.spb);
  if (grid == 0) return;
  size_t smem = (size_t)shp.spb * c.n * R * sizeof(cplx<float>);
  if (smem > 200 * 1024) throw Error(DDTM_ERR_ARG, "coarse_even: " + std::to_string(R) + " right-hand sides of " +
                                                       std::to_string(c.n) + " dofs exceed the shared-memory stage");
  set_dynamic_smem((const void*)k_coarse_even<DS, RC>, 200 * 1024);
  k_coarse_even<DS, RC><<<grid, shp.threads, smem, st>>>(t, rhs, v, c.Dc.as<DS>(), c.Dinv.as<float2>(), c.nbr_eo.as<int>(),
                                                         c.even.as<int>(), ne, c.n, R, shp.groups, sr, sh);
  CKL("coarse_even");
}

void launch_coarse_even(const CoarseLevel& c, cplx<float>* t, const cplx<float>* rhs, const cplx<float>* v, int R, float sr,
                        float sh, cudaStream_t st) {
  ScopedTimer timer_("coarse_even_f32", st, R);
  const CoarseShape shp = coarse_shape(c.n, R);
  if (shp.rc == 4) coarse_even_t<float2, 4>(c, shp, t, rhs, v, R, sr, sh, st);
  else if (shp.rc == 2) coarse_even_t<float2, 2>(c, shp, t, rhs, v, R, sr, sh, st);
  else coarse_even_t<float2, 1>(c, shp, t, rhs, v, R, sr, sh, st);
}

void launch_parity_copy(const CoarseLevel& c, int parity, cplx<float>* compact, cplx<float>* full, int R, int dir,
                        cudaStream_t st) {
  ScopedTimer timer_("parity_copy", st);
  int cnt = parity == 0 ? (int)c.h_even.size() : (int)c.h_odd.size();
  const int* list = parity == 0 ? c.even.as<int>() : c.odd.as<int>();
  size_t tot = (size_t)cnt * c.n * R;
  k_parity_copy<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(compact, full, list, cnt, c.n * R, dir);
  CKL("parity_copy");
}

void launch_coarse_interleave(const CoarseLevel& c, cplx<float>* v, double* canon, int r, int R, int dir,
                              cudaStream_t st) {
  size_t nc = (size_t)c.Nc * c.n;
  k_coarse_interleave<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(reinterpret_cast<float2*>(v), canon, nc, r, R, dir);
  CKL("coarse_interleave");
}

void launch_self_inverse(CoarseLevel& c, double mu_c, cudaStream_t st) {
  ScopedTimer timer_("self_inverse", st);
  int ne = (int)c.h_even.size();
  c.Dinv.ensure((size_t)ne * c.n * c.n * sizeof(float2));
  size_t smem = (size_t)c.n * 2 * c.n * sizeof(cplx<double>);
  int threads = ((c.n + 31) / 32) * 32;
  if (c.prec == PREC_F16) {
    // the inverses feed FP16 operator images: Gauss-Jordan in FP32 (FP64 is slow on this GPU)
    const size_t smem32 = (size_t)c.n * 2 * c.n * sizeof(cplx<float>);
    set_dynamic_smem((const void*)k_self_inverse<float2, float>, smem32);
    k_self_inverse<float2, float><<<ne, threads, smem32, st>>>(c.Dinv.as<float2>(), c.Dc.as<float2>(), c.even.as<int>(),
                                                               c.n, c.nv, mu_c);
  } else {
    set_dynamic_smem((const void*)k_self_inverse<float2, double>, smem);
    k_self_inverse<float2, double><<<ne, threads, smem, st>>>(c.Dinv.as<float2>(), c.Dc.as<float2>(), c.even.as<int>(),
                                                                c.n, c.nv, mu_c);
  }
  CKL("self_inverse");
  if (c.prec == PREC_F16) build_inverse_images(c, st);
  c.inv_mu = mu_c;
  c.inv_valid = true;
}

}  // namespace ddtm

// Gamma5-compatible aggregation (Sec. 2.3): building P from test vectors,
// restriction R = P^dagger and prolongation P.
//
// P layout (FP32 or FP16 complex): P[((blk*2 + s)*nv + i)*6*Vb + comp*Vb + loc]
// = column (blk, s, i) of P at site loc, spinor component 6 s + comp (spins
// 2s, 2s+1 x 3 colours), i.e. the chirality-s half of aggregate blk.
// Coarse vectors: complex FP32 [site][2 nv], dof s*nv + i.
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"

namespace ddtm {

__device__ __forceinline__ size_t pidx(int blk, int s, int i, int comp, int loc, int nv, int Vb) {
  return (((size_t)(blk * 2 + s) * nv + i) * 6 + comp) * Vb + loc;
}

// Gather the chirality-s halves of nv test vectors (FP32 fine fields, internal
// layout, field stride 12*V) into P and orthonormalise each aggregate half in
// index order by classical Gram-Schmidt applied twice per vector (CGS2): the
// same QR factor with positive diagonal as modified Gram-Schmidt, up to
// rounding, with one batched CTA reduction per pass instead of one per pair.
// Each thread keeps its site's 6 components in FP32; the CTA-wide inner
// products are summed over warps in FP64.  One CTA per (blk, s); thread = site.
static const int BP_CH = 8;  // inner products reduced together
__global__ void k_build_P(float2* __restrict__ P, const float2* __restrict__ tv, int nv, int Vb, long V) {
  __shared__ double red[32][2 * BP_CH];  // per warp partial sums of one chunk
  __shared__ float2 hco[64];             // projection coefficients <v_j, v_i>
  const int blk = blockIdx.x >> 1, s = blockIdx.x & 1;
  const int loc = threadIdx.x, lane = loc & 31, w = loc >> 5, nw = blockDim.x >> 5;
  const bool act = loc < Vb;
  if (act)
    for (int i = 0; i < nv; i++)
      for (int comp = 0; comp < 6; comp++)
        P[pidx(blk, s, i, comp, loc, nv, Vb)] =
            tv[(size_t)i * 12 * V + ((size_t)blk * 12 + 6 * s + comp) * Vb + loc];
  __syncthreads();
  for (int i = 0; i < nv; i++) {
    float2 vi[6];
#pragma unroll
    for (int comp = 0; comp < 6; comp++) vi[comp] = act ? P[pidx(blk, s, i, comp, loc, nv, Vb)] : make_float2(0.f, 0.f);
    for (int pass = 0; pass < 2 && i > 0; pass++) {
      // h_j = <v_j, v_i> for all j < i, in chunks of BP_CH
      for (int j0 = 0; j0 < i; j0 += BP_CH) {
        float pr[BP_CH], pi[BP_CH];
#pragma unroll
        for (int c = 0; c < BP_CH; c++) {
          pr[c] = pi[c] = 0.f;
          const int j = j0 + c;
          if (act && j < i)
#pragma unroll
            for (int comp = 0; comp < 6; comp++) {
              const float2 vj = P[pidx(blk, s, j, comp, loc, nv, Vb)];
              pr[c] += vj.x * vi[comp].x + vj.y * vi[comp].y;
              pi[c] += vj.x * vi[comp].y - vj.y * vi[comp].x;
            }
        }
#pragma unroll
        for (int c = 0; c < BP_CH; c++) {
          const float a = warp_sum(pr[c]), b = warp_sum(pi[c]);
          if (lane == 0) {
            red[w][2 * c] = a;
            red[w][2 * c + 1] = b;
          }
        }
        __syncthreads();
        if (loc < BP_CH && j0 + loc < i) {
          double a = 0, b = 0;
          for (int k = 0; k < nw; k++) {
            a += red[k][2 * loc];
            b += red[k][2 * loc + 1];
          }
          hco[j0 + loc] = make_float2((float)a, (float)b);
        }
        __syncthreads();
      }
      // v_i -= sum_j h_j v_j
      if (act)
        for (int j = 0; j < i; j++) {
          const float2 h = hco[j];
#pragma unroll
          for (int comp = 0; comp < 6; comp++) {
            const float2 vj = P[pidx(blk, s, j, comp, loc, nv, Vb)];
            vi[comp].x -= h.x * vj.x - h.y * vj.y;
            vi[comp].y -= h.x * vj.y + h.y * vj.x;
          }
        }
      __syncthreads();  // hco is rewritten by the next pass
    }
    float pn = 0;
#pragma unroll
    for (int comp = 0; comp < 6; comp++) pn += vi[comp].x * vi[comp].x + vi[comp].y * vi[comp].y;
    pn = warp_sum(pn);
    if (lane == 0) red[w][0] = pn;
    __syncthreads();
    double nn = 0;
    for (int k = 0; k < nw; k++) nn += red[k][0];
    const float inv = nn > 0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    if (act)
#pragma unroll
      for (int comp = 0; comp < 6; comp++)
        P[pidx(blk, s, i, comp, loc, nv, Vb)] = make_float2(vi[comp].x * inv, vi[comp].y * inv);
    __syncthreads();  // v_i is read by the later vectors; red is reused
  }
}

// Each CTA re-reads its aggregate half (nv x 6 x Vb complex FP32) from L2 in every Gram-Schmidt
// step; when more CTAs run at once than L2 can hold the halves of, those re-reads go to HBM.  The
// residency per SM is therefore capped (by reserving unused dynamic shared memory) so that the halves
// of all resident CTAs take about BP_L2_BYTES: 3 CTAs per SM for nv = 24 and 4^4 aggregates (at
// 32^3 x 64: 28.4 ms per build, against 29.4 ms with the 5 per SM the registers allow and 34.4 ms
// with 2 per SM, which cuts the HBM traffic tenfold but leaves too few warps to hide L2 latency).
#ifndef DDTM_BP_L2_MB
#define DDTM_BP_L2_MB 136
#endif
static const size_t BP_L2_BYTES = (size_t)DDTM_BP_L2_MB << 20;

void launch_build_P(const FineGeom& g, float2* P, const float2* tv, int nv, cudaStream_t st) {
  ScopedTimer timer_("build_P", st, nv);
  int threads = ((g.Vb + 31) / 32) * 32;
  int dev = 0, sms = 0, smem_sm = 0, smem_blk = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  CK(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  CK(cudaFuncGetAttributes(&fa, (const void*)k_build_P));
  const size_t half = (size_t)nv * 6 * g.Vb * sizeof(float2);
  size_t per_sm = (BP_L2_BYTES + half * sms / 2) / (half * (size_t)sms);  // rounded
  size_t smem = 0;
  if (per_sm < 1) per_sm = 1;
  if (per_sm < 8) {
    // at most per_sm CTAs per SM: each reserves its share of the SM's shared memory, less its
    // static shared memory and the 1 KB per CTA the runtime keeps
    smem = (size_t)smem_sm / per_sm - 1024 - fa.sharedSizeBytes;
    if (smem + fa.sharedSizeBytes > (size_t)smem_blk) smem = (size_t)smem_blk - fa.sharedSizeBytes;
    set_dynamic_smem((const void*)k_build_P, smem);
  }
  k_build_P<<<g.Nb * 2, threads, smem, st>>>(P, tv, nv, g.Vb, g.V);
  CKL("build_P");
}

template <typename PS>
__device__ __forceinline__ cplx<float> ldp(const PS* p);
template <>
__device__ __forceinline__ cplx<float> ldp<float2>(const float2* p) { return ld(p); }
template <>
__device__ __forceinline__ cplx<float> ldp<__half2>(const __half2* p) { return ld(p); }

// c = P^dagger psi per aggregate for a batch of R fine fields (field r at
// psi + r * fstride, its FP16 scales at pn + r * V); c interleaved,
// c[(blk * n + o) * R + r].  One CTA per block and chunk of RC right-hand
// sides: the RC block vectors are staged in shared memory (FP32, [rc][12][Vb]);
// warp w computes outputs o = w, w + nwarps, ... for all RC of them, lanes
// striding over sites, then warp reductions.
template <int PI, typename PS, int RC>
__global__ void k_restrict(cplx<float>* __restrict__ c, Spinor<PI> psi, size_t fstride, long V, const PS* __restrict__ P,
                           int nv, int R, int Rs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<float>* sp = reinterpret_cast<cplx<float>*>(smem_raw);
  const int Vb = psi.Vb;
  const int blk = blockIdx.x;
  const int r0 = blockIdx.y * RC;
  const int nr = R - r0 < RC ? R - r0 : RC;
  for (int rc = 0; rc < nr; rc++) {
    Spinor<PI> f = psi;
    f.d += (size_t)(r0 + rc) * fstride;
    if (f.nrm) f.nrm += (size_t)(r0 + rc) * V;
    for (int loc = threadIdx.x; loc < Vb; loc += blockDim.x) {
      cplx<typename Prec<PI>::real> v[12];
      f.load(blk, loc, v);
#pragma unroll
      for (int k = 0; k < 12; k++) sp[((size_t)rc * 12 + k) * Vb + loc] = cplx<float>((float)v[k].re, (float)v[k].im);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = 2 * nv;
  for (int o = w; o < n; o += nw) {
    int s = o / nv, i = o - s * nv;
    cplx<float> acc[RC];
#pragma unroll
    for (int rc = 0; rc < RC; rc++) acc[rc] = cplx<float>(0, 0);
    const PS* col = P + ((size_t)(blk * 2 + s) * nv + i) * 6 * Vb;
    for (int comp = 0; comp < 6; comp++)
      for (int loc = lane; loc < Vb; loc += 32) {
        cplx<float> pv = ldp<PS>(col + comp * Vb + loc);
#pragma unroll
        for (int rc = 0; rc < RC; rc++)
          if (rc < nr) cmac_conj(acc[rc], pv, sp[((size_t)rc * 12 + 6 * s + comp) * Vb + loc]);
      }
#pragma unroll
    for (int rc = 0; rc < RC; rc++) {
      acc[rc].re = warp_sum(acc[rc].re);
      acc[rc].im = warp_sum(acc[rc].im);
      if (lane == 0 && rc < nr) c[((size_t)blk * n + o) * Rs + r0 + rc] = acc[rc];
    }
  }
}

// The same restriction with P read once per HC right-hand sides (the kernel
// above reads it once per RC = 4): one CTA per block and chunk of HC
// right-hand sides works through the
// two chirality halves s in turn; for each it stages components 6s..6s+5 of the
// chunk's block vectors in shared memory (FP32, [rc][6][Vb]: 72 KB for 6
// right-hand sides at Vb = 256, so three CTAs share an SM), and warp w
// computes OW outputs of half s at once (each staged entry read once serves OW outputs, each P entry HC
// right-hand sides).  Every output is a sum over the block's 6 Vb entries in
// the same order as k_restrict (lane partial sums over sites, then a warp sum).
template <int PI, typename PS, int HC, int OW>
__global__ void __launch_bounds__(256, 3) k_restrict_half(cplx<float>* __restrict__ c, Spinor<PI> psi, size_t fstride,
                                                          long V, const PS* __restrict__ P, int nv, int R, int Rs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sp = reinterpret_cast<float2*>(smem_raw);  // [HC][6][Vb]
  const int Vb = psi.Vb, blk = blockIdx.x, r0 = blockIdx.y * HC;
  const int nr = R - r0 < HC ? R - r0 : HC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = 2 * nv;
  for (int s = 0; s < 2; s++) {
    if (s) __syncthreads();  // the previous half's reads are done
    for (int rc = 0; rc < HC; rc++) {
      Spinor<PI> f = psi;
      f.d += (size_t)(r0 + rc) * fstride;
      if (f.nrm) f.nrm += (size_t)(r0 + rc) * V;
      for (int loc = threadIdx.x; loc < Vb; loc += blockDim.x) {
        if (rc < nr) {
          cplx<typename Prec<PI>::real> v[12];
          f.load(blk, loc, v);
#pragma unroll
          for (int k = 0; k < 6; k++) {
            const cplx<typename Prec<PI>::real> a = s ? v[6 + k] : v[k];  // constant register indices
            sp[((size_t)rc * 6 + k) * Vb + loc] = make_float2((float)a.re, (float)a.im);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 6; k++) sp[((size_t)rc * 6 + k) * Vb + loc] = make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
    for (int i0 = w * OW; i0 < nv; i0 += nw * OW) {
      cplx<float> acc[OW][HC];
#pragma unroll
      for (int u = 0; u < OW; u++)
#pragma unroll
        for (int rc = 0; rc < HC; rc++) acc[u][rc] = cplx<float>(0, 0);
      for (int comp = 0; comp < 6; comp++)
        for (int loc = lane; loc < Vb; loc += 32) {
          cplx<float> pv[OW];
#pragma unroll
          for (int u = 0; u < OW; u++) {
            const int i = i0 + u < nv ? i0 + u : nv - 1;
            pv[u] = ldp<PS>(P + (((size_t)(blk * 2 + s) * nv + i) * 6 + comp) * Vb + loc);
          }
#pragma unroll
          for (int rc = 0; rc < HC; rc++) {
            const float2 f2 = sp[((size_t)rc * 6 + comp) * Vb + loc];
            const cplx<float> fv(f2.x, f2.y);
#pragma unroll
            for (int u = 0; u < OW; u++) cmac_conj(acc[u][rc], pv[u], fv);
          }
        }
#pragma unroll
      for (int u = 0; u < OW; u++)
#pragma unroll
        for (int rc = 0; rc < HC; rc++) {
          acc[u][rc].re = warp_sum(acc[u][rc].re);
          acc[u][rc].im = warp_sum(acc[u][rc].im);
          if (lane == 0 && rc < nr && i0 + u < nv) c[((size_t)blk * n + s * nv + i0 + u) * Rs + r0 + rc] = acc[u][rc];
        }
    }
  }
}

// x_r = P e_r (add = 0) or x_r += P e_r (add = 1) for a batch of R fields; e
// interleaved.  One CTA per block, thread = site; e_B (n x R) staged in shared
// memory; each P entry loaded once per thread serves RC right-hand sides.
template <int PO, typename PS, int RC>
__global__ void k_prolong(Spinor<PO> x, size_t fstride, long V, const cplx<float>* __restrict__ e, const PS* __restrict__ P,
                          int nv, int R, int Rs, int add) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<float>* se = reinterpret_cast<cplx<float>*>(smem_raw);
  typedef typename Prec<PO>::real Rl;
  const int Vb = x.Vb;
  const int blk = blockIdx.x;
  const int n = 2 * nv;
  for (int k = threadIdx.x; k < n * Rs; k += blockDim.x) se[k] = e[(size_t)blk * n * Rs + k];
  __syncthreads();
  for (int loc = threadIdx.x; loc < Vb; loc += blockDim.x) {
    for (int r0 = 0; r0 < R; r0 += RC) {
      const int nr = R - r0 < RC ? R - r0 : RC;
      cplx<float> acc[RC][12];
#pragma unroll
      for (int rc = 0; rc < RC; rc++)
#pragma unroll
        for (int k = 0; k < 12; k++) acc[rc][k] = cplx<float>(0, 0);
      for (int s = 0; s < 2; s++)
        for (int i = 0; i < nv; i++) {
          cplx<float> ev[RC];
#pragma unroll
          for (int rc = 0; rc < RC; rc++) ev[rc] = rc < nr ? se[(s * nv + i) * Rs + r0 + rc] : cplx<float>(0, 0);
          const PS* col = P + ((size_t)(blk * 2 + s) * nv + i) * 6 * Vb + loc;
#pragma unroll
          for (int comp = 0; comp < 6; comp++) {
            cplx<float> pv = ldp<PS>(col + (size_t)comp * Vb);
#pragma unroll
            for (int rc = 0; rc < RC; rc++) cmac(acc[rc][6 * s + comp], pv, ev[rc]);
          }
        }
#pragma unroll
      for (int rc = 0; rc < RC; rc++) {
        if (rc >= nr) break;
        Spinor<PO> f = x;
        f.d += (size_t)(r0 + rc) * fstride;
        if (f.nrm) f.nrm += (size_t)(r0 + rc) * V;
        cplx<Rl> out[12];
        if (add) f.loadw(blk, loc, out);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          cplx<Rl> a((Rl)acc[rc][k].re, (Rl)acc[rc][k].im);
          out[k] = add ? out[k] + a : a;
        }
        f.store(blk, loc, out);
      }
    }
  }
}

// The same prolongation with P read once per HC right-hand sides (the kernel
// above reads it once per PRO_RC = 2): one CTA per block and chunk of HC
// right-hand sides, thread = site.  The 6 x HC components of chirality half
// s = 0 are formed in registers and parked in shared memory ([HC][6][Vb],
// each thread its own site), those of s = 1 are formed next, and the site's 12
// components of each right-hand side are stored together (FP16 storage keeps
// one scale per site).  Every component is the same sum, in the same order,
// as in k_prolong, so the results are identical.
template <int PO, typename PS, int HC>
__global__ void __launch_bounds__(256, 2) k_prolong_half(Spinor<PO> x, size_t fstride, long V, const cplx<float>* __restrict__ e,
                                                         const PS* __restrict__ P, int nv, int R, int Rs, int add) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef typename Prec<PO>::real Rl;
  const int Vb = x.Vb, blk = blockIdx.x, n = 2 * nv, r0 = blockIdx.y * HC;
  const int nr = R - r0 < HC ? R - r0 : HC;
  float2* park = reinterpret_cast<float2*>(smem_raw);                       // [HC][6][Vb]
  cplx<float>* se = reinterpret_cast<cplx<float>*>(park + (size_t)HC * 6 * Vb);  // [n][HC]
  for (int k = threadIdx.x; k < n * HC; k += blockDim.x) {
    const int o = k / HC, rc = k - o * HC;
    se[k] = rc < nr ? e[((size_t)blk * n + o) * Rs + r0 + rc] : cplx<float>(0, 0);
  }
  __syncthreads();
  for (int loc = threadIdx.x; loc < Vb; loc += blockDim.x) {
#pragma unroll 1
    for (int s = 0; s < 2; s++) {
      cplx<float> acc[HC][6];
#pragma unroll
      for (int rc = 0; rc < HC; rc++)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[rc][c] = cplx<float>(0, 0);
      for (int i = 0; i < nv; i++) {
        const PS* col = P + ((size_t)(blk * 2 + s) * nv + i) * 6 * Vb + loc;
        cplx<float> pv[6];
#pragma unroll
        for (int c = 0; c < 6; c++) pv[c] = ldp<PS>(col + (size_t)c * Vb);
#pragma unroll
        for (int rc = 0; rc < HC; rc++) {
          const cplx<float> ev = se[(s * nv + i) * HC + rc];
#pragma unroll
          for (int c = 0; c < 6; c++) cmac(acc[rc][c], pv[c], ev);
        }
      }
      if (s == 0) {
#pragma unroll
        for (int rc = 0; rc < HC; rc++)
#pragma unroll
          for (int c = 0; c < 6; c++) park[((size_t)rc * 6 + c) * Vb + loc] = make_float2(acc[rc][c].re, acc[rc][c].im);
      } else {
#pragma unroll
        for (int rc = 0; rc < HC; rc++) {
          if (rc >= nr) break;
          Spinor<PO> f = x;
          f.d += (size_t)(r0 + rc) * fstride;
          if (f.nrm) f.nrm += (size_t)(r0 + rc) * V;
          cplx<Rl> out[12];
          if (add) f.loadw(blk, loc, out);
#pragma unroll
          for (int k = 0; k < 12; k++) {
            cplx<float> a;
            if (k < 6) {
              const float2 v = park[((size_t)rc * 6 + k) * Vb + loc];
              a = cplx<float>(v.x, v.y);
            } else {
              a = acc[rc][k - 6];
            }
            const cplx<Rl> ar((Rl)a.re, (Rl)a.im);
            out[k] = add ? out[k] + ar : ar;
          }
          f.store(blk, loc, out);
        }
      }
    }
  }
}

static const int RST_RC = 4, PRO_RC = 2;
static const int PH_C = 6;  // right-hand sides per CTA of k_prolong_half

static const int RH_C = 6, RH_OW = 3;  // right-hand sides per CTA, outputs per warp pass
template <int PI, typename PS>
static void restrict_p(const FineGeom& g, cplx<float>* c, Spinor<PI> f, size_t fstride, const PS* P, int nv, int R,
                       int Rs, cudaStream_t st) {
  if (R > RST_RC && (size_t)RH_C * 6 * g.Vb * sizeof(float2) <= 200 * 1024) {
    // several chunks of RST_RC would read P once per chunk: read it once per RH_C right-hand sides
    const size_t smem = (size_t)RH_C * 6 * g.Vb * sizeof(float2);
    set_dynamic_smem((const void*)k_restrict_half<PI, PS, RH_C, RH_OW>, smem);
    dim3 grid(g.Nb, (R + RH_C - 1) / RH_C);
    k_restrict_half<PI, PS, RH_C, RH_OW><<<grid, 256, smem, st>>>(c, f, fstride, g.V, P, nv, R, Rs);
    return;
  }
  size_t smem = (size_t)RST_RC * 12 * g.Vb * sizeof(cplx<float>);
  set_dynamic_smem((const void*)k_restrict<PI, PS, RST_RC>, 200 * 1024);
  dim3 grid(g.Nb, (R + RST_RC - 1) / RST_RC);
  k_restrict<PI, PS, RST_RC><<<grid, 256, smem, st>>>(c, f, fstride, g.V, P, nv, R, Rs);
}

template <typename PS>
static void restrict_t(const FineGeom& g, int pin, cplx<float>* c, const void* psi, const float* pn, const PS* P, int nv, int R,
                       int Rs, cudaStream_t st) {
  size_t fs = (size_t)g.V * 12;
  if (pin == PREC_F64) restrict_p<PREC_F64, PS>(g, c, Spinor<PREC_F64>{(double2*)psi, nullptr, g.Vb}, fs, P, nv, R, Rs, st);
  else if (pin == PREC_F32) restrict_p<PREC_F32, PS>(g, c, Spinor<PREC_F32>{(float2*)psi, nullptr, g.Vb}, fs, P, nv, R, Rs, st);
  else restrict_p<PREC_F16, PS>(g, c, Spinor<PREC_F16>{(__half2*)psi, (float*)pn, g.Vb}, fs, P, nv, R, Rs, st);
  CKL("restrict");
}

template <int PO, typename PS>
static void prolong_half_p(const FineGeom& g, Spinor<PO> x, size_t fs, const cplx<float>* e, const PS* P, int nv, int R,
                           int Rs, int add, size_t smem, cudaStream_t st) {
  set_dynamic_smem((const void*)k_prolong_half<PO, PS, PH_C>, smem);
  dim3 grid(g.Nb, (R + PH_C - 1) / PH_C);
  const int threads = g.Vb < 256 ? ((g.Vb + 31) / 32) * 32 : 256;
  k_prolong_half<PO, PS, PH_C><<<grid, threads, smem, st>>>(x, fs, g.V, e, P, nv, R, Rs, add);
}

template <typename PS>
static void prolong_t(const FineGeom& g, int pout, void* x, float* xn, const cplx<float>* e, const PS* P, int nv, int R,
                      int Rs, int add, cudaStream_t st) {
  size_t smem = (size_t)2 * nv * Rs * sizeof(cplx<float>);
  int threads = g.Vb < 128 ? ((g.Vb + 31) / 32) * 32 : 128;
  size_t fs = (size_t)g.V * 12;
  const size_t hsmem = (size_t)PH_C * 6 * g.Vb * sizeof(float2) + (size_t)2 * nv * PH_C * sizeof(cplx<float>);
  if (R > PRO_RC && pout != PREC_F64 && hsmem <= 100 * 1024) {
    // several chunks of PRO_RC would read P once per chunk: read it once per PH_C right-hand sides
    if (pout == PREC_F32)
      prolong_half_p<PREC_F32, PS>(g, Spinor<PREC_F32>{(float2*)x, nullptr, g.Vb}, fs, e, P, nv, R, Rs, add, hsmem, st);
    else
      prolong_half_p<PREC_F16, PS>(g, Spinor<PREC_F16>{(__half2*)x, xn, g.Vb}, fs, e, P, nv, R, Rs, add, hsmem, st);
    CKL("prolong");
    return;
  }
  if (pout == PREC_F64)
    k_prolong<PREC_F64, PS, PRO_RC><<<g.Nb, threads, smem, st>>>(Spinor<PREC_F64>{(double2*)x, nullptr, g.Vb}, fs, g.V, e,
                                                                 P, nv, R, Rs, add);
  else if (pout == PREC_F32)
    k_prolong<PREC_F32, PS, PRO_RC><<<g.Nb, threads, smem, st>>>(Spinor<PREC_F32>{(float2*)x, nullptr, g.Vb}, fs, g.V, e,
                                                                 P, nv, R, Rs, add);
  else
    k_prolong<PREC_F16, PS, PRO_RC><<<g.Nb, threads, smem, st>>>(Spinor<PREC_F16>{(__half2*)x, xn, g.Vb}, fs, g.V, e, P,
                                                                 nv, R, Rs, add);
  CKL("prolong");
}

void launch_restrict(const FineGeom& g, int pin, cplx<float>* c, const void* psi, const float* pn, const void* P,
                     int pprec, int nv, int R, int Rs, cudaStream_t st) {
  ScopedTimer timer_(pin == PREC_F16 ? "restrict_f16" : pin == PREC_F32 ? "restrict_f32" : "restrict_f64", st, R);
  if (pprec == PREC_F16) restrict_t<__half2>(g, pin, c, psi, pn, (const __half2*)P, nv, R, Rs, st);
  else restrict_t<float2>(g, pin, c, psi, pn, (const float2*)P, nv, R, Rs, st);
}

void launch_prolong(const FineGeom& g, int pout, void* x, float* xn, const cplx<float>* e, const void* P, int pprec,
                    int nv, int R, int Rs, int add, cudaStream_t st) {
  ScopedTimer timer_(pout == PREC_F16 ? "prolong_f16" : pout == PREC_F32 ? "prolong_f32" : "prolong_f64", st, R);
  if (pprec == PREC_F16) prolong_t<__half2>(g, pout, x, xn, e, (const __half2*)P, nv, R, Rs, add, st);
  else prolong_t<float2>(g, pout, x, xn, e, (const float2*)P, nv, R, Rs, add, st);
}

__global__ void k_P_to_half(const float2* __restrict__ P, __half2* __restrict__ Ph, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { float2 a = P[i]; Ph[i] = __floats2half2_rn(a.x, a.y); }
}

void launch_P_to_half(const float2* P, __half2* Ph, size_t n, cudaStream_t st) {
  k_P_to_half<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, Ph, n);
  CKL("P_to_half");
}

// Counter-based Gaussian draws for the random start of the setup: element i
// takes two SplitMix64 outputs (Steele, Lea, Flood 2014) of key + 2i and
// key + 2i + 1 as uniforms and maps them by Box-Muller to (re, im) ~ N(0, 1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_gaussian(float2* __restrict__ out, size_t n, uint64_t key) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double u1 = ((splitmix64(key + 2 * i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double u2 = ((splitmix64(key + 2 * i + 1) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  double r = sqrt(-2.0 * log(u1)), th = 6.283185307179586 * u2;
  out[i] = make_float2((float)(r * cos(th)), (float)(r * sin(th)));
}

void launch_gaussian(float2* out, size_t n, uint64_t key, cudaStream_t st) {
  k_gaussian<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, key);
  CKL("gaussian");
}

// P in canonical form for inspection: W[(s*nv + i)][site][spin][colour], zero
// on the other chirality.
struct CanonMapT {
  int L[4], b[4], NB[4];
  int Vb, Nb;
  const uint32_t* loc_coord;
};

__global__ void k_P_to_canon(double2* __restrict__ W, const float2* __restrict__ P, int nv, CanonMapT m) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long V = (long)m.Vb * m.Nb;
  if (s >= V) return;
  int blk = (int)(s / m.Vb), loc = (int)(s - (long)blk * m.Vb);
  int B[4], r = blk;
  B[1] = r % m.NB[1]; r /= m.NB[1];
  B[2] = r % m.NB[2]; r /= m.NB[2];
  B[3] = r % m.NB[3];
  B[0] = r / m.NB[3];
  uint32_t lc = m.loc_coord[loc];
  int t = B[0] * m.b[0] + (lc & 255), x = B[1] * m.b[1] + ((lc >> 8) & 255);
  int y = B[2] * m.b[2] + ((lc >> 16) & 255), z = B[3] * m.b[3] + ((lc >> 24) & 255);
  size_t site = (((size_t)t * m.L[3] + z) * m.L[2] + y) * m.L[1] + x;
  for (int sc = 0; sc < 2; sc++)
    for (int i = 0; i < nv; i++)
      for (int c = 0; c < 12; c++) {
        double2 v = make_double2(0, 0);
        if (c / 6 == sc) {
          float2 a = P[pidx(blk, sc, i, c - 6 * sc, loc, nv, m.Vb)];
          v = make_double2(a.x, a.y);
        }
        W[((size_t)(sc * nv + i) * V + site) * 12 + c] = v;
      }
}

void launch_P_to_canon(const FineGeom& g, double* W, const float2* P, int nv, cudaStream_t st) {
  CanonMapT m;
  for (int k = 0; k < 4; k++) { m.L[k] = g.L[k]; m.b[k] = g.b[k]; m.NB[k] = g.NB[k]; }
  m.Vb = g.Vb;
  m.Nb = g.Nb;
  m.loc_coord = g.loc_coord.as<uint32_t>();
  k_P_to_canon<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>((double2*)W, P, nv, m);
  CKL("P_to_canon");
}

}  // namespace ddtm

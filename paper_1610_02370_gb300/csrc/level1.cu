// The intermediate level of a three-level hierarchy (Sec. 2.2 K-cycle, Sec. 2.3
// recursion): aggregation of the level-1 lattice into blocks of level-1 sites,
// P_1 from level-1 test vectors (Gamma5_c-compatible: the two chirality halves
// of the level-1 dofs are orthonormalised separately, Sec. 2.3), restriction
// and prolongation between level 1 and level 2 on interleaved batches, the
// level-2 Galerkin operator D_2 = P_1^+ D_1 P_1, and the red-black SAP smoother
// on D_1 (Sec. 2.4) with minimal-residual block solves on the full block.
//
// Layouts (n1 = 2 nv0 dofs per level-1 site, nv1 level-1 test vectors):
//   interleaved batch : v[(site * n + k) * R + r]   (as every coarse vector)
//   test vectors      : tv[(i * Nc1 + site) * n1 + k]
//   P_1               : P[(((A * 2 + s) * nv1 + i) * Vb + q) * h + k], h = n1 / 2,
//                       column (s, i) of aggregate A at its q-th site, dof s*h + k
//   D_2               : the layout of every coarse operator (coarse.cu), n2 = 2 nv1.
#include <math.h>

#include "coarse.h"
#include "common.cuh"
#include "ddtm_internal.h"
#include "level1.h"
#include "timer.h"

namespace ddtm {

// ---- P_1: classical Gram-Schmidt applied twice per vector, per aggregate half -------------
// One CTA per (aggregate A, half s).  The nv1 restricted test vectors (m = Vb * h
// entries each) sit in shared memory as M[i][e]; vector i is orthogonalised
// against 0..i-1 (all coefficients from the same vector, twice), then
// normalised.  Inner products: per-thread FP32 products summed in FP64.
__global__ void k_l1_build_P(float2* __restrict__ P, const float2* __restrict__ tv, const int* __restrict__ sites,
                             int Nc1, int n1, int Vb, int nv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int h = n1 / 2, m = Vb * h;
  float2* M = reinterpret_cast<float2*>(smem_raw);            // [nv][m]
  double2* coef = reinterpret_cast<double2*>(M + (size_t)nv * m);  // [nv]
  double* red = reinterpret_cast<double*>(coef + nv);         // [2 * warps]
  const int A = blockIdx.x >> 1, s = blockIdx.x & 1;
  const int nt = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5, nw = nt >> 5;
  for (int idx = t; idx < nv * m; idx += nt) {
    const int i = idx / m, e = idx - i * m, q = e / h, k = e - q * h;
    const int site = sites[(size_t)A * Vb + q];
    M[idx] = tv[((size_t)i * Nc1 + site) * n1 + s * h + k];
  }
  __syncthreads();
  for (int i = 0; i < nv; i++) {
    float2* vi = M + (size_t)i * m;
    for (int pass = 0; pass < 2; pass++) {
      // coef[j] = <v_j, v_i>, one warp per j
      for (int j = w; j < i; j += nw) {
        const float2* vj = M + (size_t)j * m;
        double re = 0, im = 0;
        for (int e = lane; e < m; e += 32) {
          const float2 a = vj[e], b = vi[e];
          re += (double)(a.x * b.x + a.y * b.y);
          im += (double)(a.x * b.y - a.y * b.x);
        }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) coef[j] = make_double2(re, im);
      }
      __syncthreads();
      for (int e = t; e < m; e += nt) {
        double re = vi[e].x, im = vi[e].y;
        for (int j = 0; j < i; j++) {
          const double2 c = coef[j];
          const float2 a = M[(size_t)j * m + e];
          re -= c.x * a.x - c.y * a.y;
          im -= c.x * a.y + c.y * a.x;
        }
        vi[e] = make_float2((float)re, (float)im);
      }
      __syncthreads();
    }
    double nn = 0;
    for (int e = t; e < m; e += nt) nn += (double)(vi[e].x * vi[e].x + vi[e].y * vi[e].y);
    nn = warp_sum(nn);
    if (lane == 0) red[w] = nn;
    __syncthreads();
    double tot = 0;
    for (int k = 0; k < nw; k++) tot += red[k];
    const float inv = tot > 0 ? (float)(1.0 / sqrt(tot)) : 0.f;
    __syncthreads();
    for (int e = t; e < m; e += nt) vi[e] = make_float2(vi[e].x * inv, vi[e].y * inv);
    __syncthreads();
  }
  float2* out = P + ((size_t)A * 2 + s) * nv * m;
  for (int idx = t; idx < nv * m; idx += nt) out[idx] = M[idx];
}

// c[(A * n2 + s * nv + i) * R + r] = sum_{q, k} conj(P_1[A][s][i][q][k]) v[(site(A, q) * n1 + s h + k) * R + r]
// for r < Rv (the columns Rv..R-1 of c are left alone); one thread per (A, row, r)
__global__ void k_l1_restrict(float2* __restrict__ c, const float2* __restrict__ v, const float2* __restrict__ P,
                              const int* __restrict__ sites, int Nagg, int Vb, int n1, int nv, int R, int Rv) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n2 = 2 * nv, h = n1 / 2;
  if (t >= (long)Nagg * n2 * Rv) return;
  const int r = (int)(t % Rv);
  const long ar = t / Rv;
  const int row = (int)(ar % n2), A = (int)(ar / n2);
  const int s = row / nv, i = row - s * nv;
  const float2* p = P + (((size_t)A * 2 + s) * nv + i) * Vb * h;
  float re = 0, im = 0;
  for (int q = 0; q < Vb; q++) {
    const float2* vq = v + ((size_t)sites[(size_t)A * Vb + q] * n1 + s * h) * R + r;
    const float2* pq = p + (size_t)q * h;
#pragma unroll 4
    for (int k = 0; k < h; k++) {
      const float2 a = __ldg(pq + k), b = vq[(size_t)k * R];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
  }
  c[((size_t)A * n2 + row) * R + r] = make_float2(re, im);
}

// v[(site * n1 + s h + k) * R + r] (= or +=) sum_i P_1[A][s][i][q][k] c[(A * n2 + s nv + i) * R + r], r < Rv;
// one thread per (site, dof, r)
__global__ void k_l1_prolong(float2* __restrict__ v, const float2* __restrict__ c, const float2* __restrict__ P,
                             const int* __restrict__ sites, int Nagg, int Vb, int n1, int nv, int R, int Rv, int add) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int h = n1 / 2, n2 = 2 * nv;
  if (t >= (long)Nagg * Vb * n1 * Rv) return;
  const int r = (int)(t % Rv);
  long rest = t / Rv;
  const int dof = (int)(rest % n1);
  rest /= n1;
  const int q = (int)(rest % Vb), A = (int)(rest / Vb);
  const int s = dof / h, k = dof - s * h;
  const float2* p = P + (((size_t)A * 2 + s) * nv) * Vb * h + (size_t)q * h + k;
  const float2* cc = c + ((size_t)A * n2 + s * nv) * R + r;
  float re = 0, im = 0;
  for (int i = 0; i < nv; i++) {
    const float2 a = __ldg(p + (size_t)i * Vb * h), b = cc[(size_t)i * R];
    re += a.x * b.x - a.y * b.y;
    im += a.x * b.y + a.y * b.x;
  }
  float2* o = v + ((size_t)sites[(size_t)A * Vb + q] * n1 + dof) * R + r;
  if (add) {
    const float2 y = *o;
    re += y.x;
    im += y.y;
  }
  *o = make_float2(re, im);
}

// Galerkin columns: Phi[(site * n1 + s h + k) * n2 + (s nv + i)] = P_1[A(site)][s][i][q(site)][k]
// (zero elsewhere); the extra site Nc1 is all zeros (read by the masked hops)
__global__ void k_l1_columns(float2* __restrict__ Phi, const float2* __restrict__ P, const int* __restrict__ sites,
                             int Nagg, int Vb, int n1, int nv) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int h = n1 / 2, n2 = 2 * nv;
  const long Nc1 = (long)Nagg * Vb;
  if (t >= (Nc1 + 1) * n1 * n2) return;
  const int col = (int)(t % n2);
  long rest = t / n2;
  const int dof = (int)(rest % n1);
  const long u = rest / n1;  // (A, q) in aggregate order
  float2 val = make_float2(0.f, 0.f);
  long site = Nc1;
  if (u < Nc1) {
    const int A = (int)(u / Vb), q = (int)(u - (long)A * Vb);
    site = sites[u];
    const int s = dof / h, k = dof - s * h, sc = col / nv, i = col - sc * nv;
    if (s == sc) val = P[((((size_t)A * 2 + s) * nv + i) * Vb + q) * h + k];
  }
  Phi[((size_t)site * n1 + dof) * n2 + col] = val;
}

// D2[((A * 9 + d) * n2 + col) * n2 + row] = sum_{q, k} conj(P_1[A][s_row][i_row][q][k]) part[(site(A,q) * n1 + s_row h + k) * n2 + col]
__global__ void k_l1_project(float2* __restrict__ D2, const float2* __restrict__ part, const float2* __restrict__ P,
                             const int* __restrict__ sites, int Nagg, int Vb, int n1, int nv, int d) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n2 = 2 * nv, h = n1 / 2;
  if (t >= (long)Nagg * n2 * n2) return;
  const int col = (int)(t % n2);
  const long ar = t / n2;
  const int row = (int)(ar % n2), A = (int)(ar / n2);
  const int s = row / nv, i = row - s * nv;
  const float2* p = P + (((size_t)A * 2 + s) * nv + i) * Vb * h;
  double re = 0, im = 0;
  for (int q = 0; q < Vb; q++) {
    const float2* pp = part + ((size_t)sites[(size_t)A * Vb + q] * n1 + s * h) * n2 + col;
    const float2* pq = p + (size_t)q * h;
    float fre = 0, fim = 0;
    for (int k = 0; k < h; k++) {
      const float2 a = __ldg(pq + k), b = pp[(size_t)k * n2];
      fre += a.x * b.x + a.y * b.y;
      fim += a.x * b.y - a.y * b.x;
    }
    re += fre;
    im += fim;
  }
  D2[(((size_t)A * 9 + d) * n2 + col) * n2 + row] = make_float2((float)re, (float)im);
}

// ---- SAP on D_1 (Sec. 2.4): one CTA per aggregate of one colour and chunk of right-hand sides ----
// Per block B (the aggregate's Vb sites) and right-hand side r:
//   rho = b - D_1(mu) x on B (full stencil; neighbours outside B from x in global memory)
//   nmr times: p = (D_1)_BB rho (hops leaving B dropped, Dirichlet), alpha = <p, rho> / <p, p>,
//              x_B += alpha rho, rho -= alpha p
// rho and p live in shared memory as [q][k][Rch]; x is updated in place (only this CTA writes B).
// Thread task: (site q, row pair, chunk of 4 right-hand sides), as the SIMT coarse stencil.
__device__ __forceinline__ void l1_mv_rows(const float2* __restrict__ A, const float2* v, int n, int ldv, float2 acc0[4],
                                           float2 acc1[4]) {
  // acc{0,1}[c] += A[r0 + {0,1}][k] v[k * ldv + c] for a column-major n x n block at A (row r0)
#pragma unroll 4
  for (int k = 0; k < n; k++) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(A + (size_t)k * n));
    const float2* vk = v + (size_t)k * ldv;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const float2 x = vk[c];
      acc0[c].x += a.x * x.x - a.y * x.y;
      acc0[c].y += a.x * x.y + a.y * x.x;
      acc1[c].x += a.z * x.x - a.w * x.y;
      acc1[c].y += a.z * x.y + a.w * x.x;
    }
  }
}

__global__ void __launch_bounds__(256) k_l1_sap_half(float2* __restrict__ x, const float2* __restrict__ b,
                                                     const float2* __restrict__ Dc, const int* __restrict__ nbr,
                                                     const int* __restrict__ sites, const int* __restrict__ blocks,
                                                     int Nc1, int Vb, int n, int nv, int R, int Rch, float mu, int nmr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rho = reinterpret_cast<float2*>(smem_raw);      // [Vb][n][Rch]
  float2* p = rho + (size_t)Vb * n * Rch;                 // [Vb][n][Rch]
  float2* coef = p + (size_t)Vb * n * Rch;                // [Rch] alpha
  int* lsite = reinterpret_cast<int*>(coef + Rch);       // [Vb] level-1 site of q
  int* lnb = lsite + Vb;                                  // [8][Vb] local index of the hop target in B, or -1
  const int A = blocks[blockIdx.x];
  const int r0 = blockIdx.y * Rch;
  const int nt = blockDim.x, t = threadIdx.x;
  for (int q = t; q < Vb; q += nt) lsite[q] = sites[(size_t)A * Vb + q];
  __syncthreads();
  for (int e = t; e < 8 * Vb; e += nt) {
    const int k = e / Vb, q = e - k * Vb;
    const int nb = nbr[(size_t)k * Nc1 + lsite[q]];
    int loc = -1;
    for (int u = 0; u < Vb; u++)
      if (lsite[u] == nb) loc = u;
    lnb[e] = loc;
  }
  const int np = n / 2, nch = Rch / 4, ntask = Vb * np * nch;
  // 1. rho = b - D_1(mu) x on B
  for (int task = t; task < ntask; task += nt) {
    const int rp = task % np, ch = (task / np) % nch, q = task / (np * nch);
    const int site = lsite[q], r0w = 2 * rp, c0 = r0 + ch * 4;
    float2 acc0[4], acc1[4];
#pragma unroll
    for (int c = 0; c < 4; c++) acc0[c] = acc1[c] = make_float2(0.f, 0.f);
    l1_mv_rows(Dc + (size_t)site * 9 * n * n + r0w, x + (size_t)site * n * R + c0, n, R, acc0, acc1);
    for (int k = 0; k < 8; k++) {
      const int src = nbr[(size_t)k * Nc1 + site];
      l1_mv_rows(Dc + ((size_t)site * 9 + 1 + k) * n * n + r0w, x + (size_t)src * n * R + c0, n, R, acc0, acc1);
    }
    const float m0 = r0w < nv ? mu : -mu, m1 = r0w + 1 < nv ? mu : -mu;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const float2 x0 = x[((size_t)site * n + r0w) * R + c0 + c], x1 = x[((size_t)site * n + r0w + 1) * R + c0 + c];
      const float2 b0 = b[((size_t)site * n + r0w) * R + c0 + c], b1 = b[((size_t)site * n + r0w + 1) * R + c0 + c];
      // D x includes the twist i mu Gamma5_c x
      rho[((size_t)q * n + r0w) * Rch + ch * 4 + c] =
          make_float2(b0.x - (acc0[c].x - m0 * x0.y), b0.y - (acc0[c].y + m0 * x0.x));
      rho[((size_t)q * n + r0w + 1) * Rch + ch * 4 + c] =
          make_float2(b1.x - (acc1[c].x - m1 * x1.y), b1.y - (acc1[c].y + m1 * x1.x));
    }
  }
  __syncthreads();
  // 2. minimal residual steps on the block operator
  for (int it = 0; it < nmr; it++) {
    for (int task = t; task < ntask; task += nt) {
      const int rp = task % np, ch = (task / np) % nch, q = task / (np * nch);
      const int site = lsite[q], r0w = 2 * rp;
      float2 acc0[4], acc1[4];
#pragma unroll
      for (int c = 0; c < 4; c++) acc0[c] = acc1[c] = make_float2(0.f, 0.f);
      l1_mv_rows(Dc + (size_t)site * 9 * n * n + r0w, rho + (size_t)q * n * Rch + ch * 4, n, Rch, acc0, acc1);
      for (int k = 0; k < 8; k++) {
        const int lq = lnb[k * Vb + q];
        if (lq < 0) continue;  // Dirichlet: the hop leaves the block
        l1_mv_rows(Dc + ((size_t)site * 9 + 1 + k) * n * n + r0w, rho + (size_t)lq * n * Rch + ch * 4, n, Rch, acc0,
                   acc1);
      }
      const float m0 = r0w < nv ? mu : -mu, m1 = r0w + 1 < nv ? mu : -mu;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const float2 x0 = rho[((size_t)q * n + r0w) * Rch + ch * 4 + c], x1 = rho[((size_t)q * n + r0w + 1) * Rch + ch * 4 + c];
        p[((size_t)q * n + r0w) * Rch + ch * 4 + c] = make_float2(acc0[c].x - m0 * x0.y, acc0[c].y + m0 * x0.x);
        p[((size_t)q * n + r0w + 1) * Rch + ch * 4 + c] = make_float2(acc1[c].x - m1 * x1.y, acc1[c].y + m1 * x1.x);
      }
    }
    __syncthreads();
    // alpha_r = <p, rho> / <p, p>: one warp per right-hand side, FP64 sums in a fixed order
    {
      const int lane = t & 31, w = t >> 5, nw = nt >> 5;
      for (int c = w; c < Rch; c += nw) {
        double pr = 0, pi = 0, pp = 0;
        for (int e = lane; e < Vb * n; e += 32) {
          const float2 a = p[(size_t)e * Rch + c], r = rho[(size_t)e * Rch + c];
          pr += (double)(a.x * r.x + a.y * r.y);
          pi += (double)(a.x * r.y - a.y * r.x);
          pp += (double)(a.x * a.x + a.y * a.y);
        }
        pr = warp_sum(pr);
        pi = warp_sum(pi);
        pp = warp_sum(pp);
        if (lane == 0) coef[c] = pp > 0 ? make_float2((float)(pr / pp), (float)(pi / pp)) : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    for (int e = t; e < Vb * n * Rch; e += nt) {
      const int c = e % Rch, qk = e / Rch, q = qk / n, k = qk - q * n;
      const float2 al = coef[c], r = rho[e], a = p[e];
      float2* xo = x + ((size_t)lsite[q] * n + k) * R + r0 + c;
      const float2 xv = *xo;
      *xo = make_float2(xv.x + al.x * r.x - al.y * r.y, xv.y + al.x * r.y + al.y * r.x);
      rho[e] = make_float2(r.x - (al.x * a.x - al.y * a.y), r.y - (al.x * a.y + al.y * a.x));
    }
    __syncthreads();
  }
}

// sep[(r * N + e)] <-> inter[e * R + r] for r < nsep (dir 0: sep -> inter, columns nsep..R-1 set to zero;
// dir 1: inter -> sep)
__global__ void k_l1_transpose(float2* __restrict__ sep, float2* __restrict__ inter, size_t N, int nsep, int R, int dir) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * R) return;
  const size_t e = t / R;
  const int r = (int)(t - e * R);
  if (dir == 0) inter[t] = r < nsep ? sep[(size_t)r * N + e] : make_float2(0.f, 0.f);
  else if (r < nsep) sep[(size_t)r * N + e] = inter[t];
}

// ---- host ---------------------------------------------------------------------------------

void launch_l1_transpose(float2* sep, float2* inter, size_t N, int nsep, int R, int dir, cudaStream_t st) {
  const size_t n = N * R;
  if (!n) return;
  k_l1_transpose<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sep, inter, N, nsep, R, dir);
  CKL("l1_transpose");
}

static unsigned blocks_for(long n, int bd) { return (unsigned)((n + bd - 1) / bd); }

void launch_l1_build_P(Level1Agg& a, const CoarseLevel& c1, cudaStream_t st) {
  ScopedTimer timer_("l1_build_P", st, a.nv);
  const int h = c1.n / 2, m = a.Vb * h;
  const size_t smem = (size_t)a.nv * m * sizeof(float2) + a.nv * sizeof(double2) + 64 * sizeof(double);
  if (smem > 220 * 1024) throw Error(DDTM_ERR_ARG, "level-1 aggregation: nv[1] x block volume x nv[0] too large");
  set_dynamic_smem((const void*)k_l1_build_P, smem);
  a.P.ensure((size_t)a.Nagg * 2 * a.nv * m * sizeof(float2));
  k_l1_build_P<<<a.Nagg * 2, 256, smem, st>>>(a.P.as<float2>(), a.tv.as<float2>(), a.sites.as<int>(), c1.Nc, c1.n,
                                                a.Vb, a.nv);
  CKL("l1_build_P");
}

void launch_l1_restrict(const Level1Agg& a, const CoarseLevel& c1, float2* c, const float2* v, int R, int Rv,
                        cudaStream_t st) {
  ScopedTimer timer_("l1_restrict", st, Rv);
  const long n = (long)a.Nagg * 2 * a.nv * Rv;
  if (!n) return;
  k_l1_restrict<<<blocks_for(n, 256), 256, 0, st>>>(c, v, a.P.as<float2>(), a.sites.as<int>(), a.Nagg, a.Vb, c1.n,
                                                     a.nv, R, Rv);
  CKL("l1_restrict");
}

void launch_l1_prolong(const Level1Agg& a, const CoarseLevel& c1, float2* v, const float2* c, int R, int Rv, int add,
                       cudaStream_t st) {
  ScopedTimer timer_("l1_prolong", st, Rv);
  const long n = (long)a.Nagg * a.Vb * c1.n * Rv;
  if (!n) return;
  k_l1_prolong<<<blocks_for(n, 256), 256, 0, st>>>(v, c, a.P.as<float2>(), a.sites.as<int>(), a.Nagg, a.Vb, c1.n,
                                                    a.nv, R, Rv, add);
  CKL("l1_prolong");
}

// D_2 = P_1^+ D_1 P_1 (without twist): the n2 columns of P_1 as one interleaved batch Phi; part 0 =
// self blocks + hops inside the aggregate, part 1 + k = hop k where it leaves the aggregate (masked
// neighbour tables read the zero site Nc1 for every other hop); each part projected on P_1 of the
// output's aggregate gives block 0, resp. 1 + k, of D_2.
void launch_l1_galerkin(const Level1Agg& a, const CoarseLevel& c1, CoarseLevel& c2, ScratchPool& pool, cudaStream_t st) {
  ScopedTimer timer_("l1_galerkin", st);
  const int n1 = c1.n, n2 = 2 * a.nv;
  const size_t cols = (size_t)(c1.Nc + 1) * n1 * n2;
  float2* Phi = (float2*)pool.get("l1_gal_phi", cols * sizeof(float2));
  float2* part = (float2*)pool.get("l1_gal_part", cols * sizeof(float2));
  k_l1_columns<<<blocks_for((long)cols, 256), 256, 0, st>>>(Phi, a.P.as<float2>(), a.sites.as<int>(), a.Nagg, a.Vb,
                                                            n1, a.nv);
  CKL("l1_columns");
  c2.Dc.ensure((size_t)a.Nagg * 9 * n2 * n2 * sizeof(float2));
  CoarseLevel view;  // c1's operator with a masked neighbour table
  view.Nc = c1.Nc;
  view.n = n1;
  view.nv = c1.nv;
  view.Dc.p = c1.Dc.p;
  view.Dc.bytes = c1.Dc.bytes;
  try {
    for (int d = 0; d < 9; d++) {
      view.nbr.p = (void*)(a.tabs.as<int>() + (size_t)d * 8 * c1.Nc);
      if (d == 0) launch_coarse_apply_full(view, (cplx<float>*)part, (const cplx<float>*)Phi, n2, 0.0, 3, 1.f, 0.f, st);
      else launch_coarse_apply_hop(view, (cplx<float>*)part, (const cplx<float>*)Phi, n2, d - 1, st);
      k_l1_project<<<blocks_for((long)a.Nagg * n2 * n2, 256), 256, 0, st>>>(c2.Dc.as<float2>(), part, a.P.as<float2>(),
                                                                           a.sites.as<int>(), a.Nagg, a.Vb, n1, a.nv, d);
      CKL("l1_project");
    }
  } catch (...) {
    view.Dc.p = nullptr;  // borrowed, not owned
    view.nbr.p = nullptr;
    throw;
  }
  view.Dc.p = nullptr;
  view.nbr.p = nullptr;
}

void launch_l1_sap_half(const Level1Agg& a, const CoarseLevel& c1, float2* x, const float2* b, int colour, double mu,
                        int nmr, int R, cudaStream_t st) {
  ScopedTimer timer_("l1_sap_half", st, R);
  if (!a.geom || a.Nagg < 2) throw Error(DDTM_ERR_STATE, "internal: level-1 aggregates not built");
  const int n = c1.n;
  // chunks of 4 right-hand sides: a level-1 lattice has few aggregates (256 per colour at 32^3 x 64),
  // so the chunks are what fills the GPU
  const int Rch = 4;
  if (Rch < 4 || R % 4) throw Error(DDTM_ERR_ARG, "internal: level-1 SAP needs batches of a multiple of 4");
  const size_t smem = 2 * (size_t)a.Vb * n * Rch * sizeof(float2) + Rch * sizeof(float2) + 9 * (size_t)a.Vb * 4;
  if (smem > 220 * 1024) throw Error(DDTM_ERR_ARG, "level-1 SAP: block volume x dofs too large for shared memory");
  set_dynamic_smem((const void*)k_l1_sap_half, smem);
  dim3 grid(a.Nagg / 2, R / Rch);
  k_l1_sap_half<<<grid, 256, smem, st>>>(x, b, c1.Dc.as<float2>(), c1.nbr.as<int>(), a.sites.as<int>(),
                                         a.colour.as<int>() + (size_t)colour * (a.Nagg / 2), c1.Nc, a.Vb, n, c1.nv, R,
                                         Rch, (float)mu, nmr);
  CKL("l1_sap_half");
}

}  // namespace ddtm

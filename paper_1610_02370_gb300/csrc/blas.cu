// Vector kernels for the Krylov solvers (Sec. 2.5), batched over right-hand
// sides: inner products (per-thread sums in the arithmetic precision of the
// operands, FP64 across CTAs, in a fixed order), Gram-Schmidt
// multi-dots and multi-axpys (fused with the norms of the result), per-rhs
// scalings, and precision conversion of fine fields.
// Layouts and type tags are described in blas.h.
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "blas.h"
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"

// Launch shapes of the coarse Gram-Schmidt kernels, measured on the 32^3 x 64 propagator step (one
// wave of resident CTAs in every case): multi-dot over groups of DOTS_JB basis vectors with spans of
// DOTS_EPT pairs per thread (JB 4: 523 ms, 2: 540, 8: 812, 16: 2623 per step; EPT 2 and 8 slower), and
// multi-axpy with MAXPY_UNROLL basis vectors in flight (2: 675 ms, 1: 840, 4: 806, 8: 892).
#ifndef DDTM_DOTS_EPT
#define DDTM_DOTS_EPT 4
#endif
#ifndef DDTM_DOTS_JB
#define DDTM_DOTS_JB 4
#endif
#ifndef DDTM_MAXPY_UNROLL
#define DDTM_MAXPY_UNROLL 2
#endif

namespace ddtm {

static constexpr int MAXPY_UNROLL = DDTM_MAXPY_UNROLL;  // basis vectors in flight per multi-axpy step

template <typename T> __device__ __forceinline__ double2 ld2(const T* p, size_t i);
template <> __device__ __forceinline__ double2 ld2<float2>(const float2* p, size_t i) { float2 a = p[i]; return make_double2(a.x, a.y); }
template <> __device__ __forceinline__ double2 ld2<double2>(const double2* p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ double2 ld2<__half2>(const __half2* p, size_t i) { float2 a = __half22float2(p[i]); return make_double2(a.x, a.y); }
template <typename T> __device__ __forceinline__ void st2(T* p, size_t i, double re, double im);
template <> __device__ __forceinline__ void st2<float2>(float2* p, size_t i, double re, double im) { p[i] = make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ void st2<double2>(double2* p, size_t i, double re, double im) { p[i] = make_double2(re, im); }
template <> __device__ __forceinline__ void st2<__half2>(__half2* p, size_t i, double re, double im) { p[i] = __floats2half2_rn((float)re, (float)im); }

// Arithmetic precision of an operation on two vector types: FP32 when both
// are FP32 or FP16 (per-thread partial sums are then short, and every
// cross-thread reduction is FP64), FP64 otherwise.
template <typename A, typename B> struct Acc { typedef double T; };
template <> struct Acc<float2, float2> { typedef float T; };
template <> struct Acc<__half2, float2> { typedef float T; };
template <> struct Acc<float2, __half2> { typedef float T; };
template <typename T> __device__ __forceinline__ cplx<T> ldc(const float2* p, size_t i) { float2 a = p[i]; return cplx<T>((T)a.x, (T)a.y); }
template <typename T> __device__ __forceinline__ cplx<T> ldc(const double2* p, size_t i) { double2 a = p[i]; return cplx<T>((T)a.x, (T)a.y); }
template <typename T> __device__ __forceinline__ cplx<T> ldc(const __half2* p, size_t i) { float2 a = __half22float2(p[i]); return cplx<T>((T)a.x, (T)a.y); }

// Two consecutive complex entries (i = pair index) as (re0, im0, re1, im1).
__device__ __forceinline__ float4 ld_pair(const float2* p, size_t i) { return __ldg(reinterpret_cast<const float4*>(p) + i); }
__device__ __forceinline__ float4 ld_pair(const __half2* p, size_t i) {
  uint2 u = __ldg(reinterpret_cast<const uint2*>(p) + i);
  float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x)), b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// Per-rhs reduction inside a CTA for interleaved sets: thread t holds the
// partial of right-hand side t % R (blockDim is a multiple of R); thread r < R
// returns the sum over threads r, r + R, ... in that order.
__device__ __forceinline__ double2 rhs_reduce(double2 v, int R, double2* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  double2 s = make_double2(0, 0);
  if ((int)threadIdx.x < R)
    for (int m = threadIdx.x; m < (int)blockDim.x; m += R) { s.x += red[m].x; s.y += red[m].y; }
  __syncthreads();
  return s;
}

// whole-CTA sum (blockDim a multiple of 32), valid in thread 0
__device__ __forceinline__ double2 cta_reduce(double2 v, double* red) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[2 * w] = v.x; red[2 * w + 1] = v.y; }
  __syncthreads();
  double2 s = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; k++) { s.x += red[2 * k]; s.y += red[2 * k + 1]; }
  __syncthreads();
  return s;
}

// partial[(j*R + r) * G + cta] of <V_j(., r), w(., r)>
template <typename TV, typename TW, bool INTER>
__global__ void k_bdots(const TV* __restrict__ V, size_t ldv, int nvec, const TW* __restrict__ w, size_t n, int R,
                        double2* __restrict__ partial) {
  __shared__ double2 red[256];
  const int G = gridDim.x;
  if (INTER) {
    const int j = blockIdx.y;
    const size_t N = n * R, bd = blockDim.x;
    const size_t chunk = ((N + (size_t)G * bd - 1) / ((size_t)G * bd)) * bd;
    const size_t beg = (size_t)blockIdx.x * chunk, end = beg + chunk < N ? beg + chunk : N;
    const TV* vj = V + (size_t)j * ldv;
    typedef typename Acc<TV, TW>::T AT;
    AT are = 0, aim = 0;
#pragma unroll 4
    for (size_t i = beg + threadIdx.x; i < end; i += bd) {
      auto x = ldc<AT>(vj, i);
      auto y = ldc<AT>(w, i);
      are += x.re * y.re + x.im * y.im;
      aim += x.re * y.im - x.im * y.re;
    }
    double2 s = rhs_reduce(make_double2(are, aim), R, red);
    if ((int)threadIdx.x < R) partial[((size_t)j * R + threadIdx.x) * G + blockIdx.x] = s;
  } else {
    const int jr = blockIdx.y, j = jr / R, r = jr - j * R;
    const TV* a = V + (size_t)j * ldv + (size_t)r * n;
    const TW* b = w + (size_t)r * n;
    typedef typename Acc<TV, TW>::T AT;
    AT are = 0, aim = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)G * blockDim.x) {
      auto x = ldc<AT>(a, i);
      auto y = ldc<AT>(b, i);
      are += x.re * y.re + x.im * y.im;
      aim += x.re * y.im - x.im * y.re;
    }
    double2 s = cta_reduce(make_double2(are, aim), reinterpret_cast<double*>(red));
    if (threadIdx.x == 0) partial[(size_t)jr * G + blockIdx.x] = s;
  }
}

// Separate sets (one contiguous vector per right-hand side): CTA (c, g, r)
// reads its chunk of w(., r) once and forms the inner products with basis
// vectors g JB ... g JB + JB - 1 of rhs r, so w is read once per JB vectors
// (not once per vector); partial[(j R + r) G + c].
template <typename TV, typename TW, int JB>
__global__ void __launch_bounds__(256) k_bdots_sep(const TV* __restrict__ V, size_t ldv, int nvec,
                                                    const TW* __restrict__ w, size_t n, int R,
                                                    double2* __restrict__ partial) {
  __shared__ double red[8][2 * JB];  // per warp (blockDim <= 256)
  const int G = gridDim.x, j0 = blockIdx.y * JB, r = blockIdx.z, bd = blockDim.x, t = threadIdx.x;
  const int nj = nvec - j0 < JB ? nvec - j0 : JB;
  const size_t chunk = ((n + (size_t)G * bd - 1) / ((size_t)G * bd)) * bd;
  const size_t beg = (size_t)blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  const TV* Vr = V + (size_t)j0 * ldv + (size_t)r * n;
  const TW* wr = w + (size_t)r * n;
  typedef typename Acc<TV, TW>::T AT;
  AT are[JB], aim[JB];
#pragma unroll
  for (int jj = 0; jj < JB; jj++) are[jj] = aim[jj] = 0;
#pragma unroll 2
  for (size_t i = beg + t; i < end; i += bd) {
    const auto y = ldc<AT>(wr, i);
#pragma unroll
    for (int jj = 0; jj < JB; jj++) {
      if (jj < nj) {
        const auto x = ldc<AT>(Vr + (size_t)jj * ldv, i);
        are[jj] += x.re * y.re + x.im * y.im;
        aim[jj] += x.re * y.im - x.im * y.re;
      }
    }
  }
  const int wi = t >> 5, nw = bd >> 5;
#pragma unroll
  for (int jj = 0; jj < JB; jj++) {
    const double a = warp_sum((double)are[jj]), b = warp_sum((double)aim[jj]);
    if ((t & 31) == 0) {
      red[wi][2 * jj] = a;
      red[wi][2 * jj + 1] = b;
    }
  }
  __syncthreads();
  if (t < nj) {
    double a = 0, b = 0;
    for (int k = 0; k < nw; k++) {
      a += red[k][2 * t];
      b += red[k][2 * t + 1];
    }
    partial[((size_t)(j0 + t) * R + r) * G + blockIdx.x] = make_double2(a, b);
  }
}

// Interleaved FP32 sets with an even number R of right-hand sides, read in
// 16-byte pairs (two consecutive right-hand sides of one entry).  Work comes
// in spans of EPT x blockDim consecutive pairs: thread t of a CTA takes pairs
// base + t + u blockDim (u < EPT) of its span, so for each basis vector a CTA
// reads one contiguous piece of EPT x blockDim pairs (long DRAM bursts rather
// than a short segment of every vector), and a thread always holds the same
// pair of right-hand sides (blockDim and the spans are multiples of R/2).
// CTA c takes spans c, c + G, ... (G = gridDim.x, sized so that every CTA gets
// the same number of spans and one wave of resident CTAs holds them all).

// Multi-dot: CTA (c, g) sweeps its spans of w against basis vectors
// g JB ... g JB + JB - 1 and writes one partial per (vector, rhs):
// partial[(j R + r) G + c].
template <int JB, int EPT, typename TV>
__global__ void __launch_bounds__(256) k_bdots_pairs(const TV* __restrict__ V, size_t ldv, int nvec,
                                                      const float4* __restrict__ w, size_t npairs, int R,
                                                      double2* __restrict__ partial) {
  extern __shared__ float red_s[];  // [blockDim][4 JB + 1]
  const int G = gridDim.x, j0 = blockIdx.y * JB, Rh = R / 2, bd = blockDim.x, t = threadIdx.x;
  const int nj = nvec - j0 < JB ? nvec - j0 : JB;
  const size_t span = (size_t)bd * EPT;
  float acc[JB][4];
#pragma unroll
  for (int jj = 0; jj < JB; jj++) acc[jj][0] = acc[jj][1] = acc[jj][2] = acc[jj][3] = 0.f;
  for (size_t base = (size_t)blockIdx.x * span; base < npairs; base += (size_t)G * span) {
    float4 y[EPT];
    bool in[EPT];
#pragma unroll
    for (int u = 0; u < EPT; u++) {
      const size_t i = base + t + (size_t)u * bd;
      in[u] = i < npairs;
      y[u] = in[u] ? __ldg(w + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int jj = 0; jj < JB; jj++) {
      if (jj < nj) {
        const TV* vj = V + (size_t)(j0 + jj) * ldv;
#pragma unroll
        for (int u = 0; u < EPT; u++) {
          if (!in[u]) continue;
          const float4 x = ld_pair(vj, base + t + (size_t)u * bd);
          acc[jj][0] += x.x * y[u].x + x.y * y[u].y;
          acc[jj][1] += x.x * y[u].y - x.y * y[u].x;
          acc[jj][2] += x.z * y[u].z + x.w * y[u].w;
          acc[jj][3] += x.z * y[u].w - x.w * y[u].z;
        }
      }
    }
  }
  const int S = 4 * JB + 1;
#pragma unroll
  for (int jj = 0; jj < JB; jj++)
#pragma unroll
    for (int c = 0; c < 4; c++) red_s[t * S + jj * 4 + c] = acc[jj][c];
  __syncthreads();
  for (int o = t; o < nj * R; o += bd) {
    const int jj = o / R, r = o - jj * R, q = r >> 1, h = r & 1;
    float sre = 0.f, sim = 0.f;
    for (int m = q; m < bd; m += Rh) {
      sre += red_s[m * S + jj * 4 + 2 * h];
      sim += red_s[m * S + jj * 4 + 2 * h + 1];
    }
    partial[((size_t)(j0 + jj) * R + r) * G + blockIdx.x] = make_double2(sre, sim);
  }
}

// w(., r) += sign * sum_j coef[j * R + r] V_j(., r) for interleaved FP32 w with
// an even number of right-hand sides, V FP32 or FP16: CTA c takes the
// contiguous units [c U / G, (c + 1) U / G) of U = npairs / (R/2) units of R/2
// pairs (balanced to a unit, a thread always on the same pair of right-hand
// sides), one 16-byte pair of w per thread and step with the basis loop inside
// (MAXPY_UNROLL vectors in flight); optional per-rhs squared norms of the
// result in npartial[r * G + cta].  (Spans of several pairs per thread, as in
// the multi-dot, measured slower here: more registers, fewer resident CTAs.)
template <typename TV>
__global__ void __launch_bounds__(256) k_bmaxpy_pairs(float2* __restrict__ w, const TV* __restrict__ V, size_t ldv,
                                                       int nvec, const double2* __restrict__ coef, size_t npairs, int R,
                                                       float sign, double2* __restrict__ npartial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sc = reinterpret_cast<float2*>(smem_raw);  // [nvec][R], times sign
  __shared__ double2 red[256];
  const int G = gridDim.x, bd = blockDim.x, Rh = R / 2, t = threadIdx.x, q = t % Rh;
  for (int k = t; k < nvec * R; k += bd) sc[k] = make_float2(sign * (float)coef[k].x, sign * (float)coef[k].y);
  __syncthreads();
  const float4* sc4 = reinterpret_cast<const float4*>(sc);  // (coef of rhs 2q, coef of rhs 2q + 1) of vector j
  const size_t nunits = npairs / Rh;
  const size_t beg = nunits * blockIdx.x / G * Rh, end = nunits * (blockIdx.x + 1) / G * Rh;
  float4* w4 = reinterpret_cast<float4*>(w);
  float nn0 = 0.f, nn1 = 0.f;
  for (size_t i = beg + t; i < end; i += bd) {
    float4 acc = w4[i];
#pragma unroll (MAXPY_UNROLL)
    for (int j = 0; j < nvec; j++) {
      const float4 c = sc4[j * Rh + q];
      const float4 v = ld_pair(V + (size_t)j * ldv, i);
      acc.x += c.x * v.x - c.y * v.y;
      acc.y += c.x * v.y + c.y * v.x;
      acc.z += c.z * v.z - c.w * v.w;
      acc.w += c.z * v.w + c.w * v.z;
    }
    w4[i] = acc;
    nn0 += acc.x * acc.x + acc.y * acc.y;
    nn1 += acc.z * acc.z + acc.w * acc.w;
  }
  if (npartial) {
    red[threadIdx.x] = make_double2(nn0, nn1);
    __syncthreads();
    if ((int)threadIdx.x < Rh) {
      double s0 = 0, s1 = 0;
      for (int m = threadIdx.x; m < bd; m += Rh) {
        s0 += red[m].x;
        s1 += red[m].y;
      }
      npartial[(size_t)(2 * threadIdx.x) * G + blockIdx.x] = make_double2(s0, 0);
      npartial[(size_t)(2 * threadIdx.x + 1) * G + blockIdx.x] = make_double2(s1, 0);
    }
  }
}

// out[k] = sum_c partial[k * ncta + c], one CTA per k, fixed order
__global__ void k_reduce_partials(const double2* __restrict__ partial, int ncta, double2* out) {
  __shared__ double red[64];
  const int k = blockIdx.x;
  double2 acc = make_double2(0, 0);
  for (int c = threadIdx.x; c < ncta; c += blockDim.x) {
    double2 v = partial[(size_t)k * ncta + c];
    acc.x += v.x;
    acc.y += v.y;
  }
  double2 s = cta_reduce(acc, red);
  if (threadIdx.x == 0) out[k] = s;
}

// w(., r) += sign * sum_j coef[j*R + r] V_j(., r); npartial[r * G + cta] = |w(., r)|^2 partials
template <typename TV, typename TW, bool INTER>
__global__ void k_bmaxpy(TW* __restrict__ w, const TV* __restrict__ V, size_t ldv, int nvec, const double2* __restrict__ coef,
                         size_t n, int R, double sign, double2* __restrict__ npartial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sc = reinterpret_cast<double2*>(smem_raw);  // coefficients
  __shared__ double2 red[256];
  const int G = gridDim.x;
  const int r_sep = INTER ? 0 : blockIdx.y;
  const int ncoef = INTER ? nvec * R : nvec;
  for (int k = threadIdx.x; k < ncoef; k += blockDim.x) sc[k] = INTER ? coef[k] : coef[(size_t)k * R + r_sep];
  __syncthreads();
  typedef typename Acc<TV, TW>::T AT;
  AT nn = 0;  // squared norm of this thread's entries, in the arithmetic precision
  // each thread updates EPT entries spaced by the CTA size (coalesced), with
  // the basis loop outside so EPT independent loads are in flight per step
  const int EPT = 4;
  if (INTER) {
    const size_t N = n * R, span = (size_t)blockDim.x * EPT;
    const int r = threadIdx.x % R;  // blockDim and span are multiples of R
    for (size_t base = (size_t)blockIdx.x * span; base < N; base += (size_t)G * span) {
      cplx<AT> acc[EPT];
      bool in[EPT];
#pragma unroll
      for (int u = 0; u < EPT; u++) {
        size_t i = base + threadIdx.x + (size_t)u * blockDim.x;
        in[u] = i < N;
        acc[u] = in[u] ? ldc<AT>(w, i) : cplx<AT>(0, 0);
      }
#pragma unroll 2
      for (int j = 0; j < nvec; j++) {
        const TV* vj = V + (size_t)j * ldv;
        double2 c = sc[j * R + r];
        AT cr = (AT)(sign * c.x), ci = (AT)(sign * c.y);
#pragma unroll
        for (int u = 0; u < EPT; u++) {
          size_t i = base + threadIdx.x + (size_t)u * blockDim.x;
          cplx<AT> v = in[u] ? ldc<AT>(vj, i) : cplx<AT>(0, 0);
          acc[u].re += cr * v.re - ci * v.im;
          acc[u].im += cr * v.im + ci * v.re;
        }
      }
#pragma unroll
      for (int u = 0; u < EPT; u++) {
        if (!in[u]) continue;
        size_t i = base + threadIdx.x + (size_t)u * blockDim.x;
        st2(w, i, acc[u].re, acc[u].im);
        nn += acc[u].re * acc[u].re + acc[u].im * acc[u].im;
      }
    }
    if (npartial) {
      double2 s = rhs_reduce(make_double2((double)nn, 0), R, red);
      if ((int)threadIdx.x < R) npartial[(size_t)threadIdx.x * G + blockIdx.x] = s;
    }
  } else {
    TW* wr = w + (size_t)r_sep * n;
    const TV* Vr = V + (size_t)r_sep * n;
    const size_t span = (size_t)blockDim.x * EPT;
    for (size_t base = (size_t)blockIdx.x * span; base < n; base += (size_t)G * span) {
      cplx<AT> acc[EPT];
      bool in[EPT];
#pragma unroll
      for (int u = 0; u < EPT; u++) {
        size_t i = base + threadIdx.x + (size_t)u * blockDim.x;
        in[u] = i < n;
        acc[u] = in[u] ? ldc<AT>(wr, i) : cplx<AT>(0, 0);
      }
#pragma unroll 2
      for (int j = 0; j < nvec; j++) {
        const TV* vj = Vr + (size_t)j * ldv;
        double2 c = sc[j];
        AT cr = (AT)(sign * c.x), ci = (AT)(sign * c.y);
#pragma unroll
        for (int u = 0; u < EPT; u++) {
          size_t i = base + threadIdx.x + (size_t)u * blockDim.x;
          cplx<AT> v = in[u] ? ldc<AT>(vj, i) : cplx<AT>(0, 0);
          acc[u].re += cr * v.re - ci * v.im;
          acc[u].im += cr * v.im + ci * v.re;
        }
      }
#pragma unroll
      for (int u = 0; u < EPT; u++) {
        if (!in[u]) continue;
        size_t i = base + threadIdx.x + (size_t)u * blockDim.x;
        st2(wr, i, acc[u].re, acc[u].im);
        nn += acc[u].re * acc[u].re + acc[u].im * acc[u].im;
      }
    }
    if (npartial) {
      double2 s = cta_reduce(make_double2((double)nn, 0), reinterpret_cast<double*>(red));
      if (threadIdx.x == 0) npartial[(size_t)r_sep * G + blockIdx.x] = s;
    }
  }
}

// y(., r) = a[r] x(., r) + b[r] y(., r); zero coefficients skip their operand.
// Interleaved sets: blockDim and the grid stride are multiples of R, so each
// thread keeps one right-hand side; separate sets: grid.y = right-hand side.
template <typename TX, typename TY, bool INTER>
__global__ void k_baxpby(const double2* __restrict__ a, const TX* x, const double2* __restrict__ b, TY* y, size_t n, int R) {
  // arithmetic in the wider of the two storage precisions; 4 independent entries per thread and step
  typedef typename Acc<TX, TY>::T AT;
  const int r = INTER ? (int)(threadIdx.x % R) : blockIdx.y;
  const double2 ca = a[r], cb = b[r];
  const bool ra = ca.x != 0 || ca.y != 0, rb = cb.x != 0 || cb.y != 0, unit_b = cb.x == 1 && cb.y == 0;
  const AT ar = (AT)ca.x, ai = (AT)ca.y, br = (AT)cb.x, bi = (AT)cb.y;
  const size_t N = INTER ? n * R : n;
  const size_t off = INTER ? 0 : (size_t)r * n;
  const size_t bd = blockDim.x, stride = (size_t)gridDim.x * bd * 4;
  for (size_t i0 = (size_t)blockIdx.x * bd * 4 + threadIdx.x; i0 < N; i0 += stride) {
    cplx<AT> u[4], v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const size_t i = i0 + (size_t)k * bd;
      const bool in = i < N;
      u[k] = in && ra ? ldc<AT>(x, off + i) : cplx<AT>(0, 0);
      v[k] = in && rb ? ldc<AT>(y, off + i) : cplx<AT>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const size_t i = i0 + (size_t)k * bd;
      if (i >= N) break;
      AT re, im;
      if (unit_b) {  // y + a x: the common update, two fused multiply-adds per component
        re = v[k].re + ar * u[k].re - ai * u[k].im;
        im = v[k].im + ar * u[k].im + ai * u[k].re;
      } else {
        re = ar * u[k].re - ai * u[k].im + br * v[k].re - bi * v[k].im;
        im = ar * u[k].im + ai * u[k].re + br * v[k].im + bi * v[k].re;
      }
      st2(y, off + i, re, im);
    }
  }
}

// y(., r) = a[r] x(., r)  (x may equal y); layout handling as k_baxpby
template <typename TX, typename TY, bool INTER>
__global__ void k_bscale(const double2* __restrict__ a, const TX* x, TY* y, size_t n, int R) {
  typedef typename Acc<TX, TY>::T AT;
  const int r = INTER ? (int)(threadIdx.x % R) : blockIdx.y;
  const AT cr = (AT)a[r].x, ci = (AT)a[r].y;
  const size_t N = INTER ? n * R : n;
  const size_t off = INTER ? 0 : (size_t)r * n;
  const size_t bd = blockDim.x, stride = (size_t)gridDim.x * bd * 4;
  for (size_t i0 = (size_t)blockIdx.x * bd * 4 + threadIdx.x; i0 < N; i0 += stride) {
    cplx<AT> u[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const size_t i = i0 + (size_t)k * bd;
      u[k] = i < N ? ldc<AT>(x, off + i) : cplx<AT>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const size_t i = i0 + (size_t)k * bd;
      if (i < N) st2(y, off + i, cr * u[k].re - ci * u[k].im, cr * u[k].im + ci * u[k].re);
    }
  }
}

template <int PI, int PO>
__global__ void k_field_convert(Spinor<PO> out, Spinor<PI> in, long V) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  int blk = (int)(s / in.Vb), loc = (int)(s - (long)blk * in.Vb);
  cplx<typename Prec<PI>::real> a[12];
  in.loadw(blk, loc, a);
  cplx<typename Prec<PO>::real> b[12];
#pragma unroll
  for (int c = 0; c < 12; c++) b[c] = cplx<typename Prec<PO>::real>(a[c].re, a[c].im);
  out.store(blk, loc, b);
}

// ---- host side -------------------------------------------------------------------------
static int lcm32(int R) {
  int a = R, b = 32;
  while (b) { int t = a % b; a = b; b = t; }
  return R / a * 32;
}
// CTA size for interleaved sets: a multiple of both R and 32, at most 256
static int inter_block(int R) {
  int l = lcm32(R);
  if (l > 256) throw Error(DDTM_ERR_ARG, "internal: batch of " + std::to_string(R) + " right-hand sides not supported");
  return (256 / l) * l;
}
static int grid_for(size_t work, int bd, int cap) {
  size_t g = (work + (size_t)bd * 4 - 1) / ((size_t)bd * 4);
  return (int)(g < 1 ? 1 : (g > (size_t)cap ? cap : g));
}

CoefRing::~CoefRing() {
  for (int i = 0; i < SLOTS; i++)
    if (ev_used[i]) cudaEventDestroy(ev[i]);
  if (host) cudaFreeHost(host);
}

const double2* CoefRing::push(const double2* vals, size_t count, cudaStream_t st) {
  if (!host) {
    slot_elems = 8192;
    CK(cudaMallocHost(&host, SLOTS * slot_elems * sizeof(double2)));
    dev.ensure(SLOTS * slot_elems * sizeof(double2));
  }
  if (count > slot_elems) throw Error(DDTM_ERR_ARG, "internal: coefficient block too large");
  int s = next;
  next = (next + 1) % SLOTS;
  if (ev_used[s]) CK(cudaEventSynchronize(ev[s]));
  else {
    CK(cudaEventCreateWithFlags(&ev[s], cudaEventDisableTiming));
    ev_used[s] = true;
  }
  memcpy(host + s * slot_elems, vals, count * sizeof(double2));
  double2* d = dev.as<double2>() + s * slot_elems;
  CK(cudaMemcpyAsync(d, host + s * slot_elems, count * sizeof(double2), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(ev[s], st));
  return d;
}

Blas::Blas(cudaStream_t s, ScratchPool* p, CoefRing* r) : st(s), pool(p), ring(r) {}

static const double2* coef_to_device(Blas* b, const double2* vals, size_t count, const char* name) {
  if (b->ring) return b->ring->push(vals, count, b->st);
  double2* d = (double2*)b->pool->get(name, count * sizeof(double2));
  CK(cudaMemcpyAsync(d, vals, count * sizeof(double2), cudaMemcpyHostToDevice, b->st));
  CK(cudaStreamSynchronize(b->st));
  return d;
}

#define DISPATCH_TYPES(TV, TW, CALL)                                                      \
  do {                                                                                    \
    if ((TV) == 1 && (TW) == 1) { typedef float2 A; typedef float2 B; CALL; }             \
    else if ((TV) == 0 && (TW) == 0) { typedef double2 A; typedef double2 B; CALL; }      \
    else if ((TV) == 1 && (TW) == 0) { typedef float2 A; typedef double2 B; CALL; }       \
    else if ((TV) == 0 && (TW) == 1) { typedef double2 A; typedef float2 B; CALL; }       \
    else if ((TV) == 2 && (TW) == 1) { typedef __half2 A; typedef float2 B; CALL; }       \
    else if ((TV) == 1 && (TW) == 2) { typedef float2 A; typedef __half2 B; CALL; }       \
    else throw Error(DDTM_ERR_ARG, "internal: unsupported vector type combination");     \
  } while (0)

static double set_bytes(const VSet& v) {
  return (double)v.n * v.R * (v.type == 0 ? 16 : v.type == 1 ? 8 : 4);
}
static const char* fam(const VSet& w, const char* coarse, const char* fine) { return w.inter ? coarse : fine; }

// basis vectors per multi-dot CTA; pairs per thread and span of the multi-dot
static const int DOTS_JB = DDTM_DOTS_JB, DOTS_EPT = DDTM_DOTS_EPT;

// CTAs of a kernel the GPU holds at once for a block size and dynamic shared
// memory (cached per kernel and shape).
static int resident_ctas(const void* kernel, int bd, size_t smem) {
  static std::mutex m;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  const auto key = std::make_tuple(kernel, bd, smem);
  {
    std::lock_guard<std::mutex> lock(m);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int dev = 0, sms = 0, per = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, bd, smem));
  const int n = (per < 1 ? 1 : per) * sms;
  std::lock_guard<std::mutex> lock(m);
  cache[key] = n;
  return n;
}
// CTAs for S spans when each CTA of `groups` grid rows is resident at once: as many rounds of
// spans as needed, the same number of spans per CTA
static int span_grid(size_t spans, int groups, int cap) {
  const size_t per_row = (size_t)(cap / groups < 1 ? 1 : cap / groups);
  const size_t rounds = (spans + per_row - 1) / per_row;
  const size_t g = (spans + rounds - 1) / rounds;
  return (int)(g < 1 ? 1 : g);
}

template <typename TV>
static void maxpy_pairs_t(const VSet& w, const VSet& V, size_t ldv, int nvec, const double2* coef_dev, double sign,
                          double2* npart, int G, int bd, cudaStream_t st) {
  set_dynamic_smem((const void*)k_bmaxpy_pairs<TV>, 200 * 1024);
  const size_t smem = (size_t)nvec * w.R * sizeof(float2);
  k_bmaxpy_pairs<TV><<<G, bd, smem, st>>>((float2*)w.p, (const TV*)V.p, ldv, nvec, coef_dev, w.n * w.R / 2, w.R,
                                          (float)sign, npart);
  CKL("bmaxpy_pairs");
}
static void launch_maxpy_pairs(const VSet& w, const VSet& V, size_t ldv, int nvec, const double2* coef_dev,
                               double sign, double2* npart, int G, int bd, cudaStream_t st) {
  if (V.type == 2) maxpy_pairs_t<__half2>(w, V, ldv, nvec, coef_dev, sign, npart, G, bd, st);
  else maxpy_pairs_t<float2>(w, V, ldv, nvec, coef_dev, sign, npart, G, bd, st);
}
// one wave of resident CTAs, each taking at least one pair per thread (and at least one unit)
static int maxpy_pairs_grid(const VSet& w, const VSet& V, int nvec, int bd) {
  const void* k = V.type == 2 ? (const void*)k_bmaxpy_pairs<__half2> : (const void*)k_bmaxpy_pairs<float2>;
  const size_t npairs = w.n * w.R / 2, units = npairs / (size_t)(w.R / 2);
  size_t g = (size_t)resident_ctas(k, bd, (size_t)nvec * w.R * sizeof(float2)), cap = npairs / (size_t)bd;
  if (g > cap) g = cap;
  if (g > units) g = units;
  return (int)(g < 1 ? 1 : g);
}
static bool pairs_ok(const VSet& V, size_t ldv, const VSet& w) {
  return w.inter && (V.type == 1 || V.type == 2) && w.type == 1 && w.R % 2 == 0 && lcm32(w.R / 2) <= 256 &&
         ldv % 2 == 0 && ((uintptr_t)V.p & 15) == 0 && ((uintptr_t)w.p & 15) == 0;
}
static int pairs_block(const VSet& w) { return inter_block(w.R / 2); }
static size_t dots_pairs_smem(int bd) { return (size_t)bd * (4 * DOTS_JB + 1) * sizeof(float); }
static int pairs_grid(const VSet& w, const VSet& V, int bd, int nvec) {
  const void* k = V.type == 2 ? (const void*)k_bdots_pairs<DOTS_JB, DOTS_EPT, __half2>
                              : (const void*)k_bdots_pairs<DOTS_JB, DOTS_EPT, float2>;
  const size_t npairs = w.n * w.R / 2, span = (size_t)bd * DOTS_EPT;
  const int groups = (nvec + DOTS_JB - 1) / DOTS_JB;
  return span_grid((npairs + span - 1) / span, groups, resident_ctas(k, bd, dots_pairs_smem(bd)));
}
template <typename TV>
static void dots_pairs_t(const VSet& V, size_t ldv, int nvec, const VSet& w, double2* partial, int G, int bd,
                         cudaStream_t st) {
  set_dynamic_smem((const void*)k_bdots_pairs<DOTS_JB, DOTS_EPT, TV>, 64 * 1024);
  dim3 grid(G, (nvec + DOTS_JB - 1) / DOTS_JB);
  k_bdots_pairs<DOTS_JB, DOTS_EPT, TV><<<grid, bd, dots_pairs_smem(bd), st>>>(
      (const TV*)V.p, ldv, nvec, (const float4*)w.p, w.n * w.R / 2, w.R, partial);
  CKL("bdots_pairs");
}
static void launch_dots_pairs(const VSet& V, size_t ldv, int nvec, const VSet& w, double2* partial, int G, int bd,
                              cudaStream_t st) {
  if (V.type == 2) dots_pairs_t<__half2>(V, ldv, nvec, w, partial, G, bd, st);
  else dots_pairs_t<float2>(V, ldv, nvec, w, partial, G, bd, st);
}

static const int SEP_JB = 4;  // basis vectors per CTA of the separate-set multi-dot
// separate-set multi-dot: about four waves of 256-thread CTAs over the (vector group, rhs) rows,
// each CTA taking at least 4 entries per thread
static int sep_grid(const VSet& w, int bd, int nvec) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t rows = (size_t)((nvec + SEP_JB - 1) / SEP_JB) * w.R;
  size_t g = (size_t)4 * 8 * sms / rows, gmax = w.n / ((size_t)bd * 4);
  if (g > gmax) g = gmax;
  if (g > 512) g = 512;
  return (int)(g < 1 ? 1 : g);
}

void Blas::dots(const VSet& V, size_t ldv, int nvec, const VSet& w, double2* out_host) {
  ScopedTimer timer_(fam(w, "blas_dots_coarse", "blas_dots_fine"), st, nvec,
                     (V.p == w.p && nvec == 1) ? set_bytes(w) : nvec * set_bytes(V) + set_bytes(w));
  const int R = w.R;
  if (nvec <= 0) return;
  const bool pairs = pairs_ok(V, ldv, w);
  int bd = pairs ? pairs_block(w) : w.inter ? inter_block(R) : 256;
  int G = pairs ? pairs_grid(w, V, bd, nvec) : w.inter ? grid_for(w.n * R, bd, 512) : sep_grid(w, bd, nvec);
  double2* partial = (double2*)pool->get("blas_partial", (size_t)nvec * R * G * sizeof(double2));
  double2* dres = (double2*)pool->get("blas_result", (size_t)nvec * R * sizeof(double2));
  dim3 grid(G, w.inter ? nvec : nvec * R);
  if (grid.y > 65535) throw Error(DDTM_ERR_ARG, "internal: too many vectors in one inner-product batch");
  if (pairs)
    launch_dots_pairs(V, ldv, nvec, w, partial, G, bd, st);
  else if (w.inter)
    DISPATCH_TYPES(V.type, w.type,
                   (k_bdots<A, B, true><<<grid, bd, 0, st>>>((const A*)V.p, ldv, nvec, (const B*)w.p, w.n, R, partial)));
  else
    DISPATCH_TYPES(V.type, w.type,
                   (k_bdots_sep<A, B, SEP_JB><<<dim3(G, (nvec + SEP_JB - 1) / SEP_JB, R), bd, 0, st>>>(
                       (const A*)V.p, ldv, nvec, (const B*)w.p, w.n, R, partial)));
  CKL("bdots");
  k_reduce_partials<<<nvec * R, 128, 0, st>>>(partial, G, dres);
  CKL("reduce_partials");
  CK(cudaMemcpyAsync(out_host, dres, (size_t)nvec * R * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

void Blas::norms2(const VSet& a, double* out_host) {
  std::vector<double2> t(a.R);
  dots(a, 0, 1, a, t.data());
  for (int r = 0; r < a.R; r++) out_host[r] = t[r].x;
}

template <typename A, typename B, bool INTER>
static void maxpy_launch(dim3 grid, int bd, size_t smem, cudaStream_t st, B* w, const A* V, size_t ldv, int nvec,
                         const double2* dc, size_t n, int R, double sign, double2* npart) {
  set_dynamic_smem((const void*)k_bmaxpy<A, B, INTER>, 200 * 1024);
  k_bmaxpy<A, B, INTER><<<grid, bd, smem, st>>>(w, V, ldv, nvec, dc, n, R, sign, npart);
}

static int maxpy_grid(size_t work, int bd) {
  size_t g = (work + (size_t)bd * 4 - 1) / ((size_t)bd * 4);
  return (int)(g < 1 ? 1 : (g > 16384 ? 16384 : g));
}

void Blas::maxpy(const VSet& w, const VSet& V, size_t ldv, int nvec, const double2* coef_host, double sign,
                 double* norms2_host) {
  ScopedTimer timer_(fam(w, "blas_maxpy_coarse", "blas_maxpy_fine"), st, nvec, nvec * set_bytes(V) + 2 * set_bytes(w));
  const int R = w.R;
  const bool pairs = pairs_ok(V, ldv, w);
  int bd = pairs ? pairs_block(w) : w.inter ? inter_block(R) : 256;
  int G = pairs ? maxpy_pairs_grid(w, V, nvec, bd) : maxpy_grid(w.inter ? w.n * R : w.n, bd);
  const double2* dc = coef_to_device(this, coef_host, (size_t)nvec * R, "blas_coef");
  double2* npart = norms2_host ? (double2*)pool->get("blas_npartial", (size_t)R * G * sizeof(double2)) : nullptr;
  size_t smem = (size_t)(w.inter ? nvec * R : nvec) * sizeof(double2);
  if (smem > 200 * 1024) throw Error(DDTM_ERR_ARG, "internal: coefficient block too large");
  dim3 grid(G, w.inter ? 1 : R);
  if (pairs)
    launch_maxpy_pairs(w, V, ldv, nvec, dc, sign, npart, G, bd, st);
  else if (w.inter)
    DISPATCH_TYPES(V.type, w.type,
                   (maxpy_launch<A, B, true>(grid, bd, smem, st, (B*)w.p, (const A*)V.p, ldv, nvec, dc, w.n, R, sign, npart)));
  else
    DISPATCH_TYPES(V.type, w.type,
                   (maxpy_launch<A, B, false>(grid, bd, smem, st, (B*)w.p, (const A*)V.p, ldv, nvec, dc, w.n, R, sign, npart)));
  CKL("bmaxpy");
  if (norms2_host) {
    double2* dres = (double2*)pool->get("blas_nresult", (size_t)R * sizeof(double2));
    k_reduce_partials<<<R, 128, 0, st>>>(npart, G, dres);
    CKL("reduce_partials");
    std::vector<double2> t(R);
    CK(cudaMemcpyAsync(t.data(), dres, (size_t)R * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int r = 0; r < R; r++) norms2_host[r] = t[r].x;
  }
}

// 4 entries per thread and step (k_baxpby, k_bscale); at most about two waves of CTAs in all, so
// each thread strides over many steps instead of the GPU scheduling short-lived CTAs
static void elementwise_grid(const VSet& y, int* bd, dim3* grid) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const size_t cap = (size_t)16 * sms;  // CTAs in all
  if (y.inter) {
    *bd = inter_block(y.R);
    size_t g = (y.n * y.R + (size_t)*bd * 4 - 1) / ((size_t)*bd * 4);
    grid->x = (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
    grid->y = 1;
  } else {
    *bd = 256;
    size_t g = (y.n + 1023) / 1024, capr = cap / (size_t)y.R < 1 ? 1 : cap / (size_t)y.R;
    grid->x = (unsigned)(g < 1 ? 1 : (g > capr ? capr : g));
    grid->y = y.R;
  }
  grid->z = 1;
}

void Blas::axpby(const double2* a_host, const VSet& x, const double2* b_host, const VSet& y) {
  ScopedTimer timer_("blas_axpby", st, 1, set_bytes(x) + 2 * set_bytes(y));
  const int R = y.R;
  std::vector<double2> ab(2 * (size_t)R);
  for (int r = 0; r < R; r++) { ab[r] = a_host[r]; ab[R + r] = b_host[r]; }
  const double2* d = coef_to_device(this, ab.data(), 2 * (size_t)R, "blas_ab");
  int bd;
  dim3 grid;
  elementwise_grid(y, &bd, &grid);
  if (y.inter)
    DISPATCH_TYPES(x.type, y.type, (k_baxpby<A, B, true><<<grid, bd, 0, st>>>(d, (const A*)x.p, d + R, (B*)y.p, y.n, R)));
  else
    DISPATCH_TYPES(x.type, y.type, (k_baxpby<A, B, false><<<grid, bd, 0, st>>>(d, (const A*)x.p, d + R, (B*)y.p, y.n, R)));
  CKL("baxpby");
}

void Blas::dots_dev(const VSet& V, size_t ldv, int nvec, const VSet& w, double2* out_dev) {
  ScopedTimer timer_(fam(w, "blas_dots_coarse", "blas_dots_fine"), st, nvec,
                     (V.p == w.p && nvec == 1) ? set_bytes(w) : nvec * set_bytes(V) + set_bytes(w));
  const int R = w.R;
  if (nvec <= 0) return;
  const bool pairs = pairs_ok(V, ldv, w);
  int bd = pairs ? pairs_block(w) : w.inter ? inter_block(R) : 256;
  int G = pairs ? pairs_grid(w, V, bd, nvec) : w.inter ? grid_for(w.n * R, bd, 512) : sep_grid(w, bd, nvec);
  double2* partial = (double2*)pool->get("blas_partial_dev", (size_t)nvec * R * G * sizeof(double2));
  dim3 grid(G, w.inter ? nvec : nvec * R);
  if (grid.y > 65535) throw Error(DDTM_ERR_ARG, "internal: too many vectors in one inner-product batch");
  if (pairs)
    launch_dots_pairs(V, ldv, nvec, w, partial, G, bd, st);
  else if (w.inter)
    DISPATCH_TYPES(V.type, w.type,
                   (k_bdots<A, B, true><<<grid, bd, 0, st>>>((const A*)V.p, ldv, nvec, (const B*)w.p, w.n, R, partial)));
  else
    DISPATCH_TYPES(V.type, w.type,
                   (k_bdots_sep<A, B, SEP_JB><<<dim3(G, (nvec + SEP_JB - 1) / SEP_JB, R), bd, 0, st>>>(
                       (const A*)V.p, ldv, nvec, (const B*)w.p, w.n, R, partial)));
  CKL("bdots");
  k_reduce_partials<<<nvec * R, 128, 0, st>>>(partial, G, out_dev);
  CKL("reduce_partials");
}

void Blas::maxpy_dev(const VSet& w, const VSet& V, size_t ldv, int nvec, const double2* coef_dev, double sign,
                     double2* norms2_dev) {
  ScopedTimer timer_(fam(w, "blas_maxpy_coarse", "blas_maxpy_fine"), st, nvec, nvec * set_bytes(V) + 2 * set_bytes(w));
  const int R = w.R;
  const bool pairs = pairs_ok(V, ldv, w);
  int bd = pairs ? pairs_block(w) : w.inter ? inter_block(R) : 256;
  int G = pairs ? maxpy_pairs_grid(w, V, nvec, bd) : maxpy_grid(w.inter ? w.n * R : w.n, bd);
  double2* npart = norms2_dev ? (double2*)pool->get("blas_npartial_dev", (size_t)R * G * sizeof(double2)) : nullptr;
  size_t smem = (size_t)(w.inter ? nvec * R : nvec) * sizeof(double2);
  if (smem > 200 * 1024) throw Error(DDTM_ERR_ARG, "internal: coefficient block too large");
  dim3 grid(G, w.inter ? 1 : R);
  if (pairs)
    launch_maxpy_pairs(w, V, ldv, nvec, coef_dev, sign, npart, G, bd, st);
  else if (w.inter)
    DISPATCH_TYPES(V.type, w.type,
                   (maxpy_launch<A, B, true>(grid, bd, smem, st, (B*)w.p, (const A*)V.p, ldv, nvec, coef_dev, w.n, R, sign, npart)));
  else
    DISPATCH_TYPES(V.type, w.type,
                   (maxpy_launch<A, B, false>(grid, bd, smem, st, (B*)w.p, (const A*)V.p, ldv, nvec, coef_dev, w.n, R, sign, npart)));
  CKL("bmaxpy");
  if (norms2_dev) {
    k_reduce_partials<<<R, 128, 0, st>>>(npart, G, norms2_dev);
    CKL("reduce_partials");
  }
}

void Blas::scale_dev(const double2* a_dev, const VSet& x, const VSet& y) {
  ScopedTimer timer_("blas_scale", st, 1, set_bytes(x) + set_bytes(y));
  const int R = y.R;
  int bd;
  dim3 grid;
  elementwise_grid(y, &bd, &grid);
  if (y.inter)
    DISPATCH_TYPES(x.type, y.type, (k_bscale<A, B, true><<<grid, bd, 0, st>>>(a_dev, (const A*)x.p, (B*)y.p, y.n, R)));
  else
    DISPATCH_TYPES(x.type, y.type, (k_bscale<A, B, false><<<grid, bd, 0, st>>>(a_dev, (const A*)x.p, (B*)y.p, y.n, R)));
  CKL("bscale");
}

double Blas::norm2(const void* a, int t, size_t n) {
  double r;
  norms2(VSet{(void*)a, t, n, 1, true}, &r);
  return r;
}

void Blas::axpby(double2 a, const void* x, int tx, double2 b, void* y, int ty, size_t n) {
  axpby(&a, VSet{(void*)x, tx, n, 1, true}, &b, VSet{y, ty, n, 1, true});
}

// ---- Arnoldi bookkeeping kernels (one thread per system) ------------------------------
__device__ __forceinline__ cplx<double> zc2(double2 v) { return cplx<double>(v.x, v.y); }
__device__ __forceinline__ double2 zd2(cplx<double> v) { return make_double2(v.re, v.im); }

__global__ void k_arnoldi_start(ArnoldiDev a, const double2* __restrict__ nr2) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  double beta = sqrt(nr2[r].x);
  for (int i = 0; i <= a.m; i++) a.g[(size_t)r * (a.m + 1) + i] = make_double2(0, 0);
  a.g[(size_t)r * (a.m + 1)] = make_double2(beta, 0);
  a.est[r] = a.bn[r] > 0 ? beta / a.bn[r] : 0.0;
  a.scale[r] = make_double2(beta > 0 ? 1.0 / beta : 0.0, 0);
}

// Column j of R lockstep Arnoldi processes: ARB systems per CTA.  The whole
// CTA first stages the new column (h, + h2) and the previous rotations in
// shared memory with independent loads, then one thread per system runs the
// sequential rotations from shared memory.  T = float for loose tolerances
// (the rotations are a dependent chain and FP64 latency is high on this GPU),
// double otherwise.
static const int ARB = 8;
template <typename T>
__global__ void __launch_bounds__(128) k_arnoldi_step(ArnoldiDev a, int j, const double2* __restrict__ h,
                                                      const double2* __restrict__ h2, const double2* __restrict__ hn2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = a.m, R = a.R, r0 = blockIdx.x * ARB;
  const int nb = R - r0 < ARB ? R - r0 : ARB;
  cplx<T>* col = reinterpret_cast<cplx<T>*>(smem_raw);  // [ARB][j + 2]
  cplx<T>* cs = col + (size_t)ARB * (j + 2);             // [ARB][j]
  cplx<T>* sn = cs + (size_t)ARB * j;                    // [ARB][j]
  for (int k = threadIdx.x; k < (j + 1) * nb; k += blockDim.x) {
    const int i = k / nb, rr = k - i * nb;
    double2 v = h[(size_t)i * R + r0 + rr];
    if (h2) {
      const double2 v2 = h2[(size_t)i * R + r0 + rr];
      v.x += v2.x;
      v.y += v2.y;
    }
    col[(size_t)rr * (j + 2) + i] = cplx<T>((T)v.x, (T)v.y);
  }
  for (int k = threadIdx.x; k < j * nb; k += blockDim.x) {
    const int rr = k / j, i = k - rr * j;
    const double2 c = a.cs[(size_t)(r0 + rr) * m + i], sv = a.sn[(size_t)(r0 + rr) * m + i];
    cs[(size_t)rr * j + i] = cplx<T>((T)c.x, (T)c.y);
    sn[(size_t)rr * j + i] = cplx<T>((T)sv.x, (T)sv.y);
  }
  __syncthreads();
  const int rr = threadIdx.x;
  if (rr >= nb) return;
  const int r = r0 + rr;
  cplx<T>* cl = col + (size_t)rr * (j + 2);
  const cplx<T>* csr = cs + (size_t)rr * j;
  const cplx<T>* snr = sn + (size_t)rr * j;
  const double hn = sqrt(hn2[r].x);
  cl[j + 1] = cplx<T>((T)hn, 0);
  for (int i = 0; i < j; i++) {
    const cplx<T> c = csr[i], sv = snr[i];
    const cplx<T> x = cl[i], y = cl[i + 1];
    cl[i] = conj(c) * x + conj(sv) * y;
    cl[i + 1] = c * y - sv * x;
  }
  cplx<double> d((double)cl[j].re, (double)cl[j].im);
  double rho = sqrt(norm2(d) + hn * hn);
  cplx<double> c = rho > 0 ? cplx<double>(d.re / rho, d.im / rho) : cplx<double>(1, 0);
  cplx<double> sv = rho > 0 ? cplx<double>(hn / rho, 0) : cplx<double>(0, 0);
  a.cs[(size_t)r * m + j] = zd2(c);
  a.sn[(size_t)r * m + j] = zd2(sv);
  cl[j] = cplx<T>((T)rho, 0);
  cl[j + 1] = cplx<T>(0, 0);
  double2* H = a.H + (size_t)r * (m + 1) * m;
  for (int i = 0; i <= j + 1; i++) H[(size_t)i * m + j] = make_double2((double)cl[i].re, (double)cl[i].im);
  double2* g = a.g + (size_t)r * (m + 1);
  cplx<double> gj = zc2(g[j]);
  g[j + 1] = zd2(-(sv * gj));
  g[j] = zd2(conj(c) * gj);
  double e = sqrt(norm2(zc2(g[j + 1])));
  a.est[r] = a.bn[r] > 0 ? e / a.bn[r] : 0.0;
  a.scale[r] = make_double2(hn > 0 ? 1.0 / hn : 0.0, 0);
}

__global__ void k_arnoldi_solve(ArnoldiDev a, int k, double2* __restrict__ y) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  const int m = a.m, R = a.R;
  const double2* H = a.H + (size_t)r * (m + 1) * m;
  const double2* g = a.g + (size_t)r * (m + 1);
  for (int i = k - 1; i >= 0; i--) {
    cplx<double> acc = zc2(g[i]);
    for (int l = i + 1; l < k; l++) acc = acc - zc2(H[(size_t)i * m + l]) * zc2(y[(size_t)l * R + r]);
    cplx<double> d = zc2(H[(size_t)i * m + i]);
    double dn = norm2(d);
    cplx<double> q = dn > 0 ? acc * cplx<double>(d.re / dn, -d.im / dn) : cplx<double>(0, 0);
    y[(size_t)i * R + r] = zd2(q);
  }
}

void launch_arnoldi_start(const ArnoldiDev& a, const double2* nr2, cudaStream_t st) {
  k_arnoldi_start<<<(a.R + 63) / 64, 64, 0, st>>>(a, nr2);
  CKL("arnoldi_start");
}
void launch_arnoldi_step(const ArnoldiDev& a, int j, const double2* h, const double2* h2, const double2* hn2,
                         cudaStream_t st, bool fp32) {
  ScopedTimer timer_("arnoldi", st);
  const unsigned grid = (unsigned)((a.R + ARB - 1) / ARB);
  if (fp32) {
    size_t smem = (size_t)ARB * (3 * j + 2) * sizeof(cplx<float>);
    set_dynamic_smem((const void*)k_arnoldi_step<float>, 200 * 1024);
    k_arnoldi_step<float><<<grid, 128, smem, st>>>(a, j, h, h2, hn2);
  } else {
    size_t smem = (size_t)ARB * (3 * j + 2) * sizeof(cplx<double>);
    set_dynamic_smem((const void*)k_arnoldi_step<double>, 200 * 1024);
    k_arnoldi_step<double><<<grid, 128, smem, st>>>(a, j, h, h2, hn2);
  }
  CKL("arnoldi_step");
}

void launch_arnoldi_solve(const ArnoldiDev& a, int k, double2* y, cudaStream_t st) {
  k_arnoldi_solve<<<(a.R + 63) / 64, 64, 0, st>>>(a, k, y);
  CKL("arnoldi_solve");
}

void launch_field_convert(const FineGeom& g, int pin, const void* in, const float* inn, int pout, void* out, float* outn,
                          cudaStream_t st) {
  ScopedTimer timer_("field_convert", st);
  unsigned grid = (unsigned)((g.V + 127) / 128);
#define CONV(A, B, SA, SB)                                                                          \
  k_field_convert<A, B><<<grid, 128, 0, st>>>(Spinor<B>{(SB*)out, outn, g.Vb}, Spinor<A>{(SA*)in, (float*)inn, g.Vb}, g.V)
  if (pin == PREC_F64 && pout == PREC_F32) CONV(PREC_F64, PREC_F32, double2, float2);
  else if (pin == PREC_F64 && pout == PREC_F16) CONV(PREC_F64, PREC_F16, double2, __half2);
  else if (pin == PREC_F32 && pout == PREC_F64) CONV(PREC_F32, PREC_F64, float2, double2);
  else if (pin == PREC_F32 && pout == PREC_F16) CONV(PREC_F32, PREC_F16, float2, __half2);
  else if (pin == PREC_F16 && pout == PREC_F64) CONV(PREC_F16, PREC_F64, __half2, double2);
  else if (pin == PREC_F16 && pout == PREC_F32) CONV(PREC_F16, PREC_F32, __half2, float2);
  else if (pin == pout) {
    CK(cudaMemcpyAsync(out, in, (size_t)g.V * 12 * (pin == PREC_F64 ? 16 : pin == PREC_F32 ? 8 : 4),
                       cudaMemcpyDeviceToDevice, st));
    if (pin == PREC_F16) CK(cudaMemcpyAsync(outn, inn, (size_t)g.V * 4, cudaMemcpyDeviceToDevice, st));
  }
#undef CONV
  CKL("field_convert");
}

}  // namespace ddtm

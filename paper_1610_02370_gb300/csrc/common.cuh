// Device-side building blocks shared by every kernel of libddtm: complex
// arithmetic, storage precisions, field views in the internal layout, the
// chiral-basis spin projections of the Wilson hop, clover matvecs and
// deterministic block reductions.
//
// Internal fine layout (one lattice block = one aggregate = one SAP domain):
//   site s = blk * Vb + loc,  loc = parity * Vb/2 + (lexloc >> 1),
//   lexloc = ((lt*bz + lz)*by + ly)*bx + lx, blk in canonical block order.
//   spinor  : store2[(blk*12 + c)*Vb + loc], c = spin*3 + colour
//   links   : store2[((blk*4 + mu)*9 + a*3 + b)*Vb + loc]   (U_mu(x)[a][b])
//   clover  : store2[(blk*36 + k)*Vb + loc], two packed Hermitian 6x6 blocks
// A store2 holds one complex number (double2, float2 or __half2).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ddtm {

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2 };

template <typename T>
struct cplx {
  T re, im;
  __host__ __device__ cplx() {}
  __host__ __device__ cplx(T r, T i) : re(r), im(i) {}
};

template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return cplx<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return cplx<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a) { return cplx<T>(-a.re, -a.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return cplx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return cplx<T>(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return cplx<T>(a.re, -a.im); }
// a*b and conj(a)*b accumulated into c
template <typename T>
__host__ __device__ __forceinline__ void cmac(cplx<T>& c, cplx<T> a, cplx<T> b) {
  c.re = fma(a.re, b.re, fma(-a.im, b.im, c.re));
  c.im = fma(a.re, b.im, fma(a.im, b.re, c.im));
}
template <typename T>
__host__ __device__ __forceinline__ void cmac_conj(cplx<T>& c, cplx<T> a, cplx<T> b) {
  c.re = fma(a.re, b.re, fma(a.im, b.im, c.re));
  c.im = fma(a.re, b.im, fma(-a.im, b.re, c.im));
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> times_i(cplx<T> a) { return cplx<T>(-a.im, a.re); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> times_minus_i(cplx<T> a) { return cplx<T>(a.im, -a.re); }
template <typename T>
__host__ __device__ __forceinline__ T norm2(cplx<T> a) { return a.re * a.re + a.im * a.im; }

// ---- storage precisions ---------------------------------------------------
template <int P> struct Prec;
template <> struct Prec<PREC_F64> { typedef double real; typedef double2 store2; static const bool scaled = false; };
template <> struct Prec<PREC_F32> { typedef float real; typedef float2 store2; static const bool scaled = false; };
template <> struct Prec<PREC_F16> { typedef float real; typedef __half2 store2; static const bool scaled = true; };

__device__ __forceinline__ cplx<double> ld(const double2* p) { double2 v = __ldg(p); return cplx<double>(v.x, v.y); }
__device__ __forceinline__ cplx<float> ld(const float2* p) { float2 v = __ldg(p); return cplx<float>(v.x, v.y); }
__device__ __forceinline__ cplx<float> ld(const __half2* p) {
  __half2 v = __ldg(p);
  float2 f = __half22float2(v);
  return cplx<float>(f.x, f.y);
}
// plain (non-__ldg) loads for buffers written earlier in the same kernel
__device__ __forceinline__ cplx<double> ldw(const double2* p) { double2 v = *p; return cplx<double>(v.x, v.y); }
__device__ __forceinline__ cplx<float> ldw(const float2* p) { float2 v = *p; return cplx<float>(v.x, v.y); }
__device__ __forceinline__ cplx<float> ldw(const __half2* p) { float2 f = __half22float2(*p); return cplx<float>(f.x, f.y); }
__device__ __forceinline__ void st(double2* p, cplx<double> a) { *p = make_double2(a.re, a.im); }
__device__ __forceinline__ void st(float2* p, cplx<float> a) { *p = make_float2(a.re, a.im); }
__device__ __forceinline__ void st(__half2* p, cplx<float> a) { *p = __floats2half2_rn(a.re, a.im); }

// ---- geometry --------------------------------------------------------------
// loc_nbr[k*Vb + loc]: bits 0..15 neighbour local index (wrapped inside the
// block), bit 16 set when the hop leaves the block.  blk_nbr[k*Nb + blk]:
// neighbour block; bit 30 set when the hop crosses an antiperiodic t boundary.
// Hop k = 2*mu + (0 forward, 1 backward).
struct Geo {
  int Vb;        // sites per block
  int Nb;        // number of blocks
  const uint32_t* loc_nbr;
  const int* blk_nbr;
};

struct Nbr {
  int blk, loc;
  bool cross;
  bool flip;  // antiperiodic sign
};

__device__ __forceinline__ Nbr neighbour(const Geo& g, int blk, int loc, int k) {
  uint32_t e = __ldg(g.loc_nbr + k * g.Vb + loc);
  Nbr n;
  n.loc = e & 0xffff;
  n.cross = (e >> 16) & 1;
  n.flip = false;
  n.blk = blk;
  if (n.cross) {
    int b = __ldg(g.blk_nbr + k * g.Nb + blk);
    n.flip = (b >> 30) & 1;
    n.blk = b & 0x3fffffff;
  }
  return n;
}

// ---- field views -----------------------------------------------------------
template <int P>
struct Spinor {
  typedef typename Prec<P>::store2 S;
  typedef typename Prec<P>::real R;
  S* d;
  float* nrm;  // per-site scale (F16 only)
  int Vb;

  __device__ __forceinline__ void load(int blk, int loc, cplx<R> v[12]) const {
    const S* p = d + (size_t)blk * 12 * Vb + loc;
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = ld(p + (size_t)c * Vb);
    if (Prec<P>::scaled) {
      R s = __ldg(nrm + (size_t)blk * Vb + loc);
#pragma unroll
      for (int c = 0; c < 12; c++) v[c] = s * v[c];
    }
  }
  // load for buffers written in the same kernel launch (no read-only cache)
  __device__ __forceinline__ void loadw(int blk, int loc, cplx<R> v[12]) const {
    const S* p = d + (size_t)blk * 12 * Vb + loc;
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = ldw(p + (size_t)c * Vb);
    if (Prec<P>::scaled) {
      R s = nrm[(size_t)blk * Vb + loc];
#pragma unroll
      for (int c = 0; c < 12; c++) v[c] = s * v[c];
    }
  }
  __device__ __forceinline__ void store(int blk, int loc, const cplx<R> v[12]) const {
    S* p = d + (size_t)blk * 12 * Vb + loc;
    if (Prec<P>::scaled) {
      R m = 0;
#pragma unroll
      for (int c = 0; c < 12; c++) m = fmax(m, fmax(fabs(v[c].re), fabs(v[c].im)));
      nrm[(size_t)blk * Vb + loc] = (float)m;
      R inv = m > 0 ? R(1) / m : R(0);
#pragma unroll
      for (int c = 0; c < 12; c++) st(p + (size_t)c * Vb, inv * v[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 12; c++) st(p + (size_t)c * Vb, v[c]);
    }
  }
};

template <int P>
struct Links {
  typedef typename Prec<P>::store2 S;
  typedef typename Prec<P>::real R;
  const S* d;
  int Vb;
  __device__ __forceinline__ void load(int blk, int loc, int mu, cplx<R> u[9]) const {
    const S* p = d + ((size_t)blk * 4 + mu) * 9 * Vb + loc;
#pragma unroll
    for (int k = 0; k < 9; k++) u[k] = ld(p + (size_t)k * Vb);
  }
};

// Packed Hermitian 6x6 pair per site: for chirality h, slots h*18 + 0..2 hold
// the real diagonal (two reals per slot), slots h*18 + 3..17 the upper
// off-diagonal entries (i<j) in row-major order.
template <int P>
struct Clover {
  typedef typename Prec<P>::store2 S;
  typedef typename Prec<P>::real R;
  const S* d;
  int Vb;
  // y_h = S_h x_h for the two chiral halves (x, y hold 12 complex: spin*3+colour)
  __device__ __forceinline__ void apply(int blk, int loc, const cplx<R> x[12], cplx<R> y[12]) const {
    const S* p = d + (size_t)blk * 36 * Vb + loc;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const cplx<R>* xh = x + 6 * h;
      cplx<R>* yh = y + 6 * h;
      R dg[6];
#pragma unroll
      for (int k = 0; k < 3; k++) {
        cplx<R> t = ld(p + (size_t)(h * 18 + k) * Vb);
        dg[2 * k] = t.re;
        dg[2 * k + 1] = t.im;
      }
#pragma unroll
      for (int i = 0; i < 6; i++) yh[i] = dg[i] * xh[i];
      int slot = 3;
#pragma unroll
      for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
          cplx<R> u = ld(p + (size_t)(h * 18 + slot) * Vb);
          cmac(yh[i], u, xh[j]);
          cmac_conj(yh[j], u, xh[i]);
          slot++;
        }
      }
    }
  }
};

// Full complex 6x6 per chirality on the even sites of a block (inverse of the
// site-local operator for one value of mu): slot (h*36 + i*6 + j) at
// d[(blk*72 + slot)*(Vb/2) + loc], loc < Vb/2.
template <int P>
struct SiteInv {
  typedef typename Prec<P>::store2 S;
  typedef typename Prec<P>::real R;
  const S* d;
  int Vh;
  __device__ __forceinline__ void apply(int blk, int loc, const cplx<R> x[12], cplx<R> y[12]) const {
    const S* p = d + (size_t)blk * 72 * Vh + loc;
#pragma unroll
    for (int h = 0; h < 2; h++) {
#pragma unroll
      for (int i = 0; i < 6; i++) {
        cplx<R> acc(0, 0);
#pragma unroll
        for (int j = 0; j < 6; j++) cmac(acc, ld(p + (size_t)(h * 36 + i * 6 + j) * Vh), x[6 * h + j]);
        y[6 * h + i] = acc;
      }
    }
  }
};

// ---- Wilson hop in the chiral basis ----------------------------------------
// gamma_0 = [[0, 1], [1, 0]], gamma_k = [[0, i s_k], [-i s_k, 0]] in 2x2 spin
// blocks, k = 1, 2, 3 for x, y, z.  (1 -/+ gamma_mu) psi has upper half h and
// lower half R h, so a hop costs one half-spinor (2 spins x 3 colours):
//   forward  (1 - gamma_mu): h = u - G l,  lower = G h
//   backward (1 + gamma_mu): h = u + G l,  lower = -G h
// with G = 1 for mu = 0 and G = i s_k for mu = k (G^2 = -1 for k, +1 for 0).
template <typename R>
__device__ __forceinline__ void apply_G(int mu, const cplx<R> a0, const cplx<R> a1, cplx<R>& b0, cplx<R>& b1) {
  if (mu == 0) {
    b0 = a0; b1 = a1;
  } else if (mu == 1) {          // i s_1 (a0, a1) = (i a1, i a0)
    b0 = times_i(a1); b1 = times_i(a0);
  } else if (mu == 2) {          // i s_2 (a0, a1) = (a1, -a0)
    b0 = a1; b1 = -a0;
  } else {                        // i s_3 (a0, a1) = (i a0, -i a1)
    b0 = times_i(a0); b1 = times_minus_i(a1);
  }
}

// h = upper half of (1 - gamma_mu) psi (fwd) or (1 + gamma_mu) psi (backward)
template <typename R>
__device__ __forceinline__ void project(int mu, bool fwd, const cplx<R> p[12], cplx<R> h[6]) {
  // u = spins 0,1 ; l = spins 2,3 ; colour index c
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cplx<R> g0, g1;
    apply_G<R>(mu, p[6 + c], p[9 + c], g0, g1);
    if (fwd) { h[c] = p[c] - g0; h[3 + c] = p[3 + c] - g1; }
    else { h[c] = p[c] + g0; h[3 + c] = p[3 + c] + g1; }
  }
}

// acc += (w, lower(w)): the full spinor whose upper half is w, with
//   forward : mu = 0 -> lower = -w,  mu = k -> lower =  i s_k w
//   backward: mu = 0 -> lower = +w,  mu = k -> lower = -i s_k w
template <typename R>
__device__ __forceinline__ void reconstruct(int mu, bool fwd, const cplx<R> w[6], cplx<R> acc[12]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[c] = acc[c] + w[c];
    acc[3 + c] = acc[3 + c] + w[3 + c];
    cplx<R> g0, g1;
    apply_G<R>(mu, w[c], w[3 + c], g0, g1);
    bool neg = (mu == 0) ? fwd : !fwd;
    if (neg) { acc[6 + c] = acc[6 + c] - g0; acc[9 + c] = acc[9 + c] - g1; }
    else { acc[6 + c] = acc[6 + c] + g0; acc[9 + c] = acc[9 + c] + g1; }
  }
}

// w = U h (colour) for both spins of the half spinor
template <typename R>
__device__ __forceinline__ void mul_U(const cplx<R> u[9], const cplx<R> h[6], cplx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cplx<R> acc(0, 0);
#pragma unroll
      for (int b = 0; b < 3; b++) cmac(acc, u[a * 3 + b], h[3 * s + b]);
      w[3 * s + a] = acc;
    }
}
// w = U^dagger h
template <typename R>
__device__ __forceinline__ void mul_Udag(const cplx<R> u[9], const cplx<R> h[6], cplx<R> w[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cplx<R> acc(0, 0);
#pragma unroll
      for (int b = 0; b < 3; b++) cmac_conj(acc, u[b * 3 + a], h[3 * s + b]);
      w[3 * s + a] = acc;
    }
}

// ---- reductions --------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ddtm

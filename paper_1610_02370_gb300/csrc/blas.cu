// Vector kernels for the Krylov solvers (Sec. 2.5): inner products with FP64
// accumulation and a deterministic two-stage reduction (fixed grid, fixed
// summation order), Gram-Schmidt multi-dots and multi-axpys, and element-wise
// updates.  Vectors are plain complex arrays (float2 or double2); fine fields
// of the internal layout qualify as they are.  FP16 fine fields are converted
// per site by k_field_convert.
#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"
#include "blas.h"

namespace ddtm {

static const int RED_GRID = 1024;  // CTAs of every reduction's first stage
static const int RED_T = 256;

template <typename T> __device__ __forceinline__ double2 ld2(const T* p, size_t i);
template <> __device__ __forceinline__ double2 ld2<float2>(const float2* p, size_t i) { float2 a = p[i]; return make_double2(a.x, a.y); }
template <> __device__ __forceinline__ double2 ld2<double2>(const double2* p, size_t i) { return p[i]; }
template <typename T> __device__ __forceinline__ void st2(T* p, size_t i, double re, double im);
template <> __device__ __forceinline__ void st2<float2>(float2* p, size_t i, double re, double im) { p[i] = make_float2((float)re, (float)im); }
template <> __device__ __forceinline__ void st2<double2>(double2* p, size_t i, double re, double im) { p[i] = make_double2(re, im); }

__device__ __forceinline__ void block_reduce2(double& a, double& b, double* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = 0;
    for (int k = 0; k < nw; k++) { a += red[2 * k]; b += red[2 * k + 1]; }
  }
  __syncthreads();
}

// partial[cta] = sum over this CTA's grid-stride elements of conj(a) b
template <typename TA, typename TB>
__global__ void k_dot_partial(const TA* __restrict__ a, const TB* __restrict__ b, size_t n, double2* partial) {
  __shared__ double red[64];
  double re = 0, im = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 x = ld2(a, i), y = ld2(b, i);
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  block_reduce2(re, im, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = make_double2(re, im);
}

// out[k] = sum_c partial[k * ncta + c], one CTA per k, fixed order
__global__ void k_reduce_partials(const double2* __restrict__ partial, int ncta, double2* out) {
  __shared__ double red[64];
  const int k = blockIdx.x;
  double re = 0, im = 0;
  for (int c = threadIdx.x; c < ncta; c += blockDim.x) {
    double2 v = partial[(size_t)k * ncta + c];
    re += v.x;
    im += v.y;
  }
  block_reduce2(re, im, red);
  if (threadIdx.x == 0) out[k] = make_double2(re, im);
}

// Multi-dot: partial[k][cta] = conj(V_k) . w over one contiguous chunk per CTA,
// w read once per chunk into shared memory.
template <typename TV, typename TW>
__global__ void k_multidot_partial(const TV* __restrict__ V, size_t ldv, int nvec, const TW* __restrict__ w, size_t n,
                                   double2* partial) {
  __shared__ double red[64];
  __shared__ double2 sw[2048];
  size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  size_t beg = (size_t)blockIdx.x * chunk, end = beg + chunk < n ? beg + chunk : n;
  for (int k = 0; k < nvec; k++) {
    double re = 0, im = 0;
    for (size_t base = beg; base < end; base += 2048) {
      size_t lim = end - base < 2048 ? end - base : 2048;
      __syncthreads();
      for (size_t t = threadIdx.x; t < lim; t += blockDim.x) sw[t] = ld2(w, base + t);
      __syncthreads();
      const TV* vk = V + (size_t)k * ldv + base;
      for (size_t t = threadIdx.x; t < lim; t += blockDim.x) {
        double2 x = ld2(vk, t), y = sw[t];
        re += x.x * y.x + x.y * y.y;
        im += x.x * y.y - x.y * y.x;
      }
    }
    block_reduce2(re, im, red);
    if (threadIdx.x == 0) partial[(size_t)k * gridDim.x + blockIdx.x] = make_double2(re, im);
  }
}

// w -= sum_k h[k] V_k     (h complex FP64 on the device)
template <typename TV, typename TW>
__global__ void k_multi_axpy(TW* __restrict__ w, const TV* __restrict__ V, size_t ldv, int nvec, const double2* h,
                             size_t n, double sign) {
  __shared__ double2 sh[256];
  for (int k = threadIdx.x; k < nvec; k += blockDim.x) sh[k] = h[k];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 acc = ld2(w, i);
    for (int k = 0; k < nvec; k++) {
      double2 v = ld2(V + (size_t)k * ldv, i), c = sh[k];
      acc.x += sign * (c.x * v.x - c.y * v.y);
      acc.y += sign * (c.x * v.y + c.y * v.x);
    }
    st2(w, i, acc.x, acc.y);
  }
}

// y = a x + b y  (a, b complex FP64; x, y may differ in type).  A zero
// coefficient means the operand is not read at all, so b = 0 assigns y = a x
// even where y holds uninitialised memory.
template <typename TX, typename TY>
__global__ void k_axpby(double2 a, const TX* x, double2 b, TY* y, size_t n) {
  const bool ra = a.x != 0 || a.y != 0, rb = b.x != 0 || b.y != 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 u = ra ? ld2(x, i) : make_double2(0, 0), v = rb ? ld2(y, i) : make_double2(0, 0);
    double re = a.x * u.x - a.y * u.y + b.x * v.x - b.y * v.y;
    double im = a.x * u.y + a.y * u.x + b.x * v.y + b.y * v.x;
    st2(y, i, re, im);
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

static unsigned stream_grid(size_t n) {
  size_t g = (n + 255) / 256;
  return (unsigned)(g < 8192 ? (g ? g : 1) : 8192);
}

// ---- host wrappers ---------------------------------------------------------------
Blas::Blas(cudaStream_t s, ScratchPool* pool) : st(s), pool(pool) {}

void Blas::dots(const void* V, int tv, size_t ldv, int nvec, const void* w, int tw, size_t n, double2* out_host) {
  ScopedTimer timer_("blas_dots", st);
  int grid = RED_GRID;
  double2* partial = (double2*)pool->get("blas_partial", (size_t)nvec * grid * sizeof(double2));
  double2* dres = (double2*)pool->get("blas_result", (size_t)nvec * sizeof(double2));
  if (nvec == 1) {
    if (tv == 1 && tw == 1) k_dot_partial<float2, float2><<<grid, RED_T, 0, st>>>((const float2*)V, (const float2*)w, n, partial);
    else if (tv == 0 && tw == 0) k_dot_partial<double2, double2><<<grid, RED_T, 0, st>>>((const double2*)V, (const double2*)w, n, partial);
    else if (tv == 1 && tw == 0) k_dot_partial<float2, double2><<<grid, RED_T, 0, st>>>((const float2*)V, (const double2*)w, n, partial);
    else k_dot_partial<double2, float2><<<grid, RED_T, 0, st>>>((const double2*)V, (const float2*)w, n, partial);
  } else {
    if (tv == 1 && tw == 1) k_multidot_partial<float2, float2><<<grid, RED_T, 0, st>>>((const float2*)V, ldv, nvec, (const float2*)w, n, partial);
    else if (tv == 0 && tw == 0) k_multidot_partial<double2, double2><<<grid, RED_T, 0, st>>>((const double2*)V, ldv, nvec, (const double2*)w, n, partial);
    else throw Error(DDTM_ERR_ARG, "internal: mixed multidot");
  }
  CKL("dot_partial");
  k_reduce_partials<<<nvec, RED_T, 0, st>>>(partial, grid, dres);
  CKL("reduce_partials");
  CK(cudaMemcpyAsync(out_host, dres, nvec * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
}

double Blas::norm2(const void* a, int t, size_t n) {
  double2 r;
  dots(a, t, 0, 1, a, t, n, &r);
  return r.x;
}

void Blas::multi_axpy(void* w, int tw, const void* V, int tv, size_t ldv, int nvec, const double2* h_host, size_t n,
                      double sign) {
  ScopedTimer timer_("blas_multi_axpy", st);
  if (nvec <= 0) return;
  if (nvec > 256) throw Error(DDTM_ERR_ARG, "internal: multi_axpy limited to 256 vectors");
  double2* dh = (double2*)pool->get("blas_coef", 256 * sizeof(double2));
  CK(cudaMemcpyAsync(dh, h_host, nvec * sizeof(double2), cudaMemcpyHostToDevice, st));
  unsigned grid = stream_grid(n);
  if (tw == 1 && tv == 1) k_multi_axpy<float2, float2><<<grid, 256, 0, st>>>((float2*)w, (const float2*)V, ldv, nvec, dh, n, sign);
  else if (tw == 0 && tv == 0) k_multi_axpy<double2, double2><<<grid, 256, 0, st>>>((double2*)w, (const double2*)V, ldv, nvec, dh, n, sign);
  else if (tw == 0 && tv == 1) k_multi_axpy<float2, double2><<<grid, 256, 0, st>>>((double2*)w, (const float2*)V, ldv, nvec, dh, n, sign);
  else k_multi_axpy<double2, float2><<<grid, 256, 0, st>>>((float2*)w, (const double2*)V, ldv, nvec, dh, n, sign);
  CKL("multi_axpy");
  // the coefficient buffer is reused by the next call: keep host and device ordered
  CK(cudaStreamSynchronize(st));
}

void Blas::axpby(double2 a, const void* x, int tx, double2 b, void* y, int ty, size_t n) {
  ScopedTimer timer_("blas_axpby", st);
  unsigned grid = stream_grid(n);
  if (tx == 1 && ty == 1) k_axpby<float2, float2><<<grid, 256, 0, st>>>(a, (const float2*)x, b, (float2*)y, n);
  else if (tx == 0 && ty == 0) k_axpby<double2, double2><<<grid, 256, 0, st>>>(a, (const double2*)x, b, (double2*)y, n);
  else if (tx == 1 && ty == 0) k_axpby<float2, double2><<<grid, 256, 0, st>>>(a, (const float2*)x, b, (double2*)y, n);
  else k_axpby<double2, float2><<<grid, 256, 0, st>>>(a, (const double2*)x, b, (float2*)y, n);
  CKL("axpby");
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

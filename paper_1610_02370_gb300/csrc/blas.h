// Host interface of the Krylov vector kernels (blas.cu).  Type tags: 0 =
// double2 (FP64 complex), 1 = float2 (FP32 complex).  Lengths n count complex
// elements; ldv is the distance in elements between consecutive vectors of a
// basis.  Results that come back to the host synchronise the stream.
#pragma once

#include "ddtm_internal.h"

namespace ddtm {

struct Blas {
  cudaStream_t st;
  ScratchPool* pool;
  Blas(cudaStream_t s, ScratchPool* pool);
  // out[k] = <V_k, w> = sum conj(V_k) w for k < nvec (FP64 accumulation)
  void dots(const void* V, int tv, size_t ldv, int nvec, const void* w, int tw, size_t n, double2* out_host);
  double norm2(const void* a, int t, size_t n);
  // w += sign * sum_k h[k] V_k
  void multi_axpy(void* w, int tw, const void* V, int tv, size_t ldv, int nvec, const double2* h_host, size_t n,
                  double sign);
  // y = a x + b y
  void axpby(double2 a, const void* x, int tx, double2 b, void* y, int ty, size_t n);
};

void launch_field_convert(const FineGeom& g, int pin, const void* in, const float* inn, int pout, void* out, float* outn,
                          cudaStream_t st);

}  // namespace ddtm

// Arithmetic peaks of the device the library runs on, measured with CUDA
// events: FP32 and FP64 fused multiply-add throughput of the SIMT units.  The
// roofline of the ALU-bound kernels (SAP block solves, Galerkin products,
// Gram-Schmidt of the aggregation, the FP64 stencil) is taken against these.
#include <cuda_runtime.h>

#include "ddtm_internal.h"

namespace ddtm {

// CHAINS independent FMA chains per thread, ITERS steps each; the result is
// written only when it equals an impossible value, so nothing is elided.
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_peak(T* sink, int iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < CHAINS; k++) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; k++) s += x[k];
  if (s == (T)-12345.678) sink[0] = s;
}

template <typename T>
static double fma_peak(int sms, double* ms_out) {
  const int chains = 8, threads = 256, ctas = sms * 8;
  const int iters = sizeof(T) == 8 ? 256 : 4096;
  T* sink = nullptr;
  CK(cudaMalloc(&sink, sizeof(T)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 6; rep++) {
    CK(cudaEventRecord(e0, 0));
    k_fma_peak<T, 8><<<ctas, threads>>>(sink, iters, (T)0.999999, (T)1e-7);
    CKL("fma_peak");
    CK(cudaEventRecord(e1, 0));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep >= 2 && ms < best) best = ms;  // first launches are warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *ms_out = best;
  double flops = 2.0 * chains * (double)iters * threads * ctas;
  return flops / (best * 1e-3);
}

}  // namespace ddtm

using namespace ddtm;

extern "C" int ddtm_measure_fma_peak(int prec, double* flops_per_s, double* ms, int* sm_count) {
  if (!flops_per_s || (prec != DDTM_PREC_F64 && prec != DDTM_PREC_F32)) return DDTM_ERR_ARG;
  try {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double t = 0;
    *flops_per_s = prec == DDTM_PREC_F64 ? fma_peak<double>(sms, &t) : fma_peak<float>(sms, &t);
    if (ms) *ms = t;
    if (sm_count) *sm_count = sms;
  } catch (const Error& e) {
    return e.code;
  } catch (const std::exception&) {
    return DDTM_ERR_CUDA;
  }
  return DDTM_OK;
}

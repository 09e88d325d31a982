// Host interface of the aggregation and coarse-level kernels (transfer.cu, coarse.cu).
#pragma once

#include "common.cuh"
#include "ddtm_internal.h"

namespace ddtm {

void build_faces(const FineGeom& g, FaceDev& faces);

// transfer.cu
void launch_build_P(const FineGeom& g, float2* P, const float2* tv, int nv, cudaStream_t st);
// R fine fields (stride 12 V complex numbers, FP16 scales stride V) <-> R coarse vectors
// interleaved with stride Rs >= R (entries r >= R of the coarse side are left alone)
void launch_restrict(const FineGeom& g, int pin, cplx<float>* c, const void* psi, const float* pn, const void* P,
                     int pprec, int nv, int R, int Rs, cudaStream_t st);
void launch_prolong(const FineGeom& g, int pout, void* x, float* xn, const cplx<float>* e, const void* P, int pprec,
                    int nv, int R, int Rs, int add, cudaStream_t st);
void launch_P_to_half(const float2* P, __half2* Ph, size_t n, cudaStream_t st);
void launch_gaussian(float2* out, size_t n, uint64_t key, cudaStream_t st);
void launch_P_to_canon(const FineGeom& g, double* W, const float2* P, int nv, cudaStream_t st);

// coarse.cu
void launch_galerkin(const FineGeom& g, const FaceDev& faces, int dprec, void* Dc, const float2* P, const void* links32,
                     const void* clover32, int nv, cudaStream_t st);
// Batched coarse vectors: R right-hand sides interleaved, v[(site * n + k) * R + r].
// full-lattice vectors: y = sy*y + sres * (mode&1: self + i mu_c Gamma5_c, mode&2: hops) x
void launch_coarse_apply_full(const CoarseLevel& c, cplx<float>* y, const cplx<float>* x, int R, double mu_c, int mode,
                              float sres, float sy, cudaStream_t st);
// parity-compact: odd outputs, self term from x_o (compact odd), hops from x_e (compact even)
void launch_coarse_apply_odd(const CoarseLevel& c, cplx<float>* y_o, const cplx<float>* x_o, const cplx<float>* x_e, int R,
                             double mu_c, int mode, float sres, float sy, cudaStream_t st);
// t_e = Dinv (sr rhs_e + sh hops(v_o)) on even sites (compact); rhs or v may be null
void launch_coarse_even(const CoarseLevel& c, cplx<float>* t, const cplx<float>* rhs, const cplx<float>* v, int R, float sr,
                        float sh, cudaStream_t st);
// dir 0: compact = full restricted to one parity; dir 1: scatter compact into full
void launch_parity_copy(const CoarseLevel& c, int parity, cplx<float>* compact, cplx<float>* full, int R, int dir,
                        cudaStream_t st);
void launch_self_inverse(CoarseLevel& c, double mu_c, cudaStream_t st);

}  // namespace ddtm

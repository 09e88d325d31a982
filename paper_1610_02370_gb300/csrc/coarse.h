// Host interface of the aggregation and coarse-level kernels (transfer.cu, coarse.cu).
#pragma once

#include <string>

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
// rows_fp16: the rows of P enter the projections rounded to FP16 (for FP16 coarse storage)
void launch_galerkin(const FineGeom& g, const FaceDev& faces, int dprec, void* Dc, const float2* P, const void* links32,
                     const void* clover32, int nv, bool rows_fp16, cudaStream_t st);
// Batched coarse vectors: R right-hand sides interleaved, v[(site * n + k) * R + r].
// full-lattice vectors: y = sy*y + sres * (mode&1: self + i mu_c Gamma5_c, mode&2: hops) x
void launch_coarse_apply_full(const CoarseLevel& c, cplx<float>* y, const cplx<float>* x, int R, double mu_c, int mode,
                              float sres, float sy, cudaStream_t st);
// y = hop `hop` (0..7) of the stencil alone, through the neighbour table c.nbr
void launch_coarse_apply_hop(const CoarseLevel& c, cplx<float>* y, const cplx<float>* x, int R, int hop, cudaStream_t st);
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
// canonical FP64 coarse vector <-> column r of an interleaved FP32 batch of R (dir 0: in, 1: out)
void launch_coarse_interleave(const CoarseLevel& c, cplx<float>* v, double* canon, int r, int R, int dir,
                              cudaStream_t st);

// coarse_tc.cu: the stencil on tensor cores, FP16 operands and FP32 accumulation.
// Operands are "images": FP16 copies laid out as the MMA reads them from shared
// memory (matrix images of the n x n blocks, vector images of R right-hand
// sides per site); see coarse_tc.cu.
struct TcGeom {
  int n, R, kpad, sbo, arows, a_bytes, ngj, b_bytes;
};
TcGeom tc_geom(int n, int R);
bool tc_supported(int n);
// Dct: matrix images of the 9 blocks of every site (from Dc)
void build_coarse_images(CoarseLevel& c, cudaStream_t st);
// Dhopt: images of D_ee^-1(e) A_d(e) for the 8 hop blocks of every even site e (from Dinv and Dc), so
// that one pass forms D_ee^-1 D_eo x of the even-odd reduced operator
void build_inverse_images(CoarseLevel& c, cudaStream_t st);
size_t tc_vector_image_bytes(const CoarseLevel& c, int nsites, int R);
// x: interleaved batch of type tag x_type (1 FP32, 2 FP16)
void launch_vector_image(const CoarseLevel& c, void* img, const void* x, int x_type, int nsites, int R, cudaStream_t st);
// One stencil pass over output slots idx < nout:
//   acc = [self] A_self(idx) X_self(idx) + [hops] sum_d A_d(site or idx) X_hop(tab[d-1][idx])
//   y  = sy * yin + sres * (acc + i mu_c Gamma5_c xs)   (FP32, if y)
//   yt = FP16 vector image of the same value            (if yt)
struct TcPass {
  const char* name;
  bool self = false, hops = false;
  const void* A_self = nullptr;
  size_t a_self_stride = 0;
  bool self_by_site = false;  // A_self indexed by osite[idx] (else by idx)
  const void* A_hop = nullptr;
  bool hop_by_slot = false;   // hop d of slot idx at A_hop + (idx * 8 + d - 1) (else (site * 9 + d)) blocks
  const void* X_self = nullptr;
  const void* X_hop = nullptr;
  const int* tab = nullptr;
  const int* osite = nullptr;
  int nout = 0;
  cplx<float>* y = nullptr;
  const cplx<float>* yin = nullptr;
  const void* xs = nullptr;  // self vector for the twist, type tag xs_type (1 FP32, 2 FP16)
  int xs_type = 1;
  float sy = 0.f, sres = 1.f, mu_c = 0.f;
  void* yt = nullptr;
};
void launch_coarse_tc(const CoarseLevel& c, const TcPass& p, int R, cudaStream_t st);
// autotuner of the tensor-core pass residency (process-wide): switch, and the
// choices made so far as JSON {shape: {"ctas_per_sm": k, "ms": [t1, t2, ...]}}
void tc_autotune_enable(bool on);
void tc_set_forced_wait_ns(uint64_t ns);
uint64_t tc_forced_wait_ns();
std::string tc_autotune_report();
// throws DDTM_ERR_TIMEOUT if a tensor-core pass gave up waiting (and clears the flag)
void check_tc_error(CoarseLevel& c);

}  // namespace ddtm

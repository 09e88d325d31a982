// Coarse stencil on the 5th-generation tensor cores (Sec. 2.3): for a batch of
// R right-hand sides,
//   y(x) = sum over items (self block, 8 hop blocks) A_d(x) v(x + d),
// with FP16 operands and FP32 accumulation, as used by the even-odd reduced
// coarsest solve (Sec. 2.5).
//
// Complex to real.  A complex n x n block A and an n x R block of vectors v
// become one real product D = A'' B with
//   A''[2i + c][k] = (c ? Im : Re) A[i][k]        (2n x n)
//   B[k][2r + b]   = (b ? Im : Re) v[k][r]        (n x 2R)
// and the epilogue combines  Re y[i][r] = D[2i][2r] - D[2i+1][2r+1],
//                            Im y[i][r] = D[2i][2r+1] + D[2i+1][2r].
// This costs exactly the 8 n^2 R real flops of the complex product; the MMA
// shape is M = 128 (2n <= 128 rows used) and N = 2R rounded up to 16.
//
// Images.  Every operand lives in HBM already in the shared-memory layout the
// MMA reads (K-major, no swizzle): element (row, k) of an image at byte
//   (row / 8) * sbo + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2,
// sbo = 16 kpad, kpad = n rounded up to 16 (padding entries are zero).  A
// matrix image holds the rows of A'' (a_bytes each); a vector image the 2R
// columns of B for one site (b_bytes each).  One pipeline stage is then two
// 1-D bulk copies (TMA engine) completing on one mbarrier.
//
// Kernel.  Persistent, two CTAs per SM (one for batches wider than 16
// right-hand sides), 6 warps: warp 0 issues the bulk copies of each
// (site, item) into a ring of stages, one thread of warp 1 issues the
// MMAs (accumulating a site's items in tensor memory, two accumulator buffers),
// warps 2-5 read the accumulator rows back (tcgen05.ld), combine real and
// imaginary parts, add the twist and the axpby terms and store FP32 and/or the
// FP16 image of the result for the next product.  Every wait is bounded; a
// timeout stops the CTA cleanly and sets *err.
#include <cuda_fp16.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <atomic>

#include "coarse.h"
#include "common.cuh"
#include "ddtm_internal.h"
#include "tc_ptx.cuh"
#include "timer.h"

namespace ddtm {

static const int TC_MAXNS = 24;          // pipeline stages at most
// Dynamic shared memory per CTA.  One issuing thread per CTA caps a CTA near
// 4-5 TB/s of bulk copies across the GPU, so two CTAs share each SM (each with
// a shorter ring) where the epilogue's registers allow it.
static const int TC_SMEM_1 = 200 * 1024;
static const int TC_SMEM_2 = 108 * 1024;
static const int TC_SMEM_3 = 70 * 1024;
// the register budget of a column-group count allows this many CTAs per SM
__host__ __device__ constexpr int tc_ctas_per_sm(int ngj) { return ngj <= 4 ? 2 : 1; }
static int tc_smem_budget(int cps) { return cps >= 3 ? TC_SMEM_3 : cps == 2 ? TC_SMEM_2 : TC_SMEM_1; }
static const uint64_t TC_WAIT_NS = 2000000000ull;
// Test hook of the timeout path: when non-zero, every pass's MMA thread first waits this long on a
// barrier that nothing completes (the wait runs out, the pass aborts, the API reports a timeout).
static std::atomic<uint64_t> g_forced_wait_ns{0};

__host__ __device__ __forceinline__ size_t img_off(int row, int k, int sbo) {
  return (size_t)(row >> 3) * sbo + (size_t)(k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

TcGeom tc_geom(int n, int R) {
  TcGeom t;
  t.n = n;
  t.R = R;
  t.kpad = (n + 15) / 16 * 16;
  t.sbo = 16 * t.kpad;
  t.arows = (2 * n + 7) / 8 * 8;
  t.a_bytes = t.arows / 8 * t.sbo;
  t.ngj = (2 * R + 7) / 8;
  t.b_bytes = t.ngj * t.sbo;
  return t;
}

bool tc_supported(int n) { return n >= 2 && 2 * n <= 128; }

// ---- image builders --------------------------------------------------------------------------
// Matrix images of column-major complex n x n blocks src[b][k][i]; one thread per
// (block, row of A'', 8-wide k group).
__global__ void k_matrix_image(char* __restrict__ img, const float2* __restrict__ src, size_t nblocks, int n, int arows,
                               int kpad, int sbo, int a_bytes) {
  const int kg = kpad / 8;
  const size_t per = (size_t)arows * kg;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nblocks * per) return;
  const size_t b = t / per;
  const int rem = (int)(t - b * per), row = rem % arows, h = rem / arows;
  __align__(16) __half v[8];
#pragma unroll
  for (int kk = 0; kk < 8; kk++) {
    const int k = 8 * h + kk;
    float f = 0.f;
    if (k < n && row < 2 * n) {
      const float2 z = __ldg(src + (b * n + k) * n + (row >> 1));
      f = (row & 1) ? z.y : z.x;
    }
    v[kk] = __float2half_rn(f);
  }
  *reinterpret_cast<uint4*>(img + b * a_bytes + img_off(row, 8 * h, sbo)) = *reinterpret_cast<const uint4*>(v);
}

__device__ __forceinline__ float2 ld_f2(const float2* p, size_t i) { return __ldg(p + i); }
__device__ __forceinline__ float2 ld_f2(const __half2* p, size_t i) { return __half22float2(p[i]); }

// Vector images of interleaved complex vectors x[(s * n + k) * R + r] (FP32 or
// FP16); one thread per (site, column j = 2r + b, 8-wide k group).
template <typename TX>
__global__ void k_vector_image(char* __restrict__ img, const TX* __restrict__ x, int nsites, int n, int R, int kpad,
                               int sbo, int ngj, int b_bytes) {
  const int kg = kpad / 8, jc = 8 * ngj;
  const size_t per = (size_t)jc * kg;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nsites * per) return;
  const size_t s = t / per;
  const int rem = (int)(t - s * per), j = rem % jc, h = rem / jc;
  const int r = j >> 1;
  __align__(16) __half v[8];
#pragma unroll
  for (int kk = 0; kk < 8; kk++) {
    const int k = 8 * h + kk;
    float f = 0.f;
    if (k < n && r < R) {
      const float2 z = ld_f2(x, (s * n + k) * R + r);
      f = (j & 1) ? z.y : z.x;
    }
    v[kk] = __float2half_rn(f);
  }
  *reinterpret_cast<uint4*>(img + s * b_bytes + img_off(j, 8 * h, sbo)) = *reinterpret_cast<const uint4*>(v);
}

// ---- the tensor-core stencil -----------------------------------------------------------------
struct TcArgs {
  const char* A_self;   // self item of output slot idx: A_self + key * a_self_stride, key = osite[idx] or idx
  size_t a_self_stride;
  int self_by_site;
  const char* A_hop;    // hop item d = 1..8 of site s: A_hop + (s * 9 + d) * a_bytes (hop_by_slot: (idx * 8 + d - 1))
  int hop_by_slot;
  const char* X_self;   // vector image of the self item: X_self + idx * b_bytes
  const char* X_hop;    // hop item d: X_hop + tab[(d - 1) * nout + idx] * b_bytes
  const int* tab;
  const int* osite;
  int nout, self, hops;
  float2* y;            // y = sy * yin + sres * (acc + i mu_c Gamma5_c xs)   (FP32, optional)
  const float2* yin;
  const void* xs;
  int xs_half;
  float sy, sres, mu_c;
  char* yt;             // FP16 image of the same result (optional)
  int n, nv, R, r0, Rk; // columns r0 .. r0 + Rk - 1 of R right-hand sides
  int kpad, sbo, a_bytes, b_bytes, ngj_all, bslot, apad, ns, nmma, tcols;
  uint32_t idesc;
  int* err;
  uint64_t forced_wait_ns;  // > 0: the MMA thread first waits this long on a barrier nothing completes
};

template <int NGJ>
__global__ void __launch_bounds__(192, tc_ctas_per_sm(NGJ)) k_coarse_tc(const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * TC_MAXNS + 6];
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sA = (ptx::smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sB = sA + (uint32_t)(a.ns * a.a_bytes + a.apad);
  const uint32_t bar0 = ptx::smem_u32(bars);
  const uint32_t FULL = bar0, EMPTY = bar0 + 8u * TC_MAXNS, ACCF = bar0 + 16u * TC_MAXNS, ACCE = ACCF + 16u,
                 FIN = ACCF + 32u, NEVER = ACCF + 40u;
  volatile int* abort_flag = &abort_sh;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.ns; s++) {
      ptx::mbar_init(FULL + 8u * s, 1);
      ptx::mbar_init(EMPTY + 8u * s, 1);
    }
    for (int b = 0; b < 2; b++) {
      ptx::mbar_init(ACCF + 8u * b, 1);
      ptx::mbar_init(ACCE + 8u * b, 4);
    }
    ptx::mbar_init(FIN, 1);
    ptx::mbar_init(NEVER, 1);  // no thread arrives on it
    abort_sh = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_sh), (uint32_t)a.tcols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_sh;

  const int G = gridDim.x;
  const int nq = (int)blockIdx.x < a.nout ? (a.nout - 1 - (int)blockIdx.x) / G + 1 : 0;
  const int ni = a.self + 8 * a.hops;

  if (warp == 0) {
    // ---- producer: bulk copies of the A and B images of every (site, item) ----
    uint32_t it = 0;
    const size_t xoff = (size_t)(a.r0 / 4) * a.sbo;
    const uint32_t xbytes = (uint32_t)(NGJ * a.sbo), stage_tx = (uint32_t)a.a_bytes + xbytes;
    for (int q = 0; q < nq; q++) {
      if (*abort_flag) break;
      const int idx = (int)blockIdx.x + q * G;
      int v = 0;
      if (lane < 8) v = a.hops ? __ldg(a.tab + (size_t)lane * a.nout + idx) : 0;
      else if (lane == 8) v = a.osite ? __ldg(a.osite + idx) : idx;
      int src[8];
#pragma unroll
      for (int d = 0; d < 8; d++) src[d] = __shfl_sync(0xffffffffu, v, d);
      const int site = __shfl_sync(0xffffffffu, v, 8);
      if (lane == 0) {
        for (int t = 0; t < ni; t++) {
          const int s = (int)(it % (uint32_t)a.ns);
          const uint32_t ph = (it / (uint32_t)a.ns) & 1u;
          if (!ptx::mbar_wait(EMPTY + 8u * s, ph ^ 1u, abort_flag, TC_WAIT_NS)) break;
          const char *Ag, *Xg;
          if (a.self && t == 0) {
            Ag = a.A_self + (size_t)(a.self_by_site ? site : idx) * a.a_self_stride;
            Xg = a.X_self + (size_t)idx * a.b_bytes + xoff;
          } else {
            const int d = t - a.self + 1;
            Ag = a.A_hop + (a.hop_by_slot ? (size_t)idx * 8 + (d - 1) : (size_t)site * 9 + d) * a.a_bytes;
            Xg = a.X_hop + (size_t)src[d - 1] * a.b_bytes + xoff;
          }
          ptx::mbar_arrive_expect_tx(FULL + 8u * s, stage_tx);
          ptx::bulk_g2s(sA + (uint32_t)(s * a.a_bytes), Ag, (uint32_t)a.a_bytes, FULL + 8u * s);
          ptx::bulk_g2s(sB + (uint32_t)(s * a.bslot), Xg, xbytes, FULL + 8u * s);
          it++;
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      // tail: every stage issued has landed (abort) or has been released by its MMAs
      // (a stage released by its MMAs has landed; once a release wait gives up, the copies of that
      // stage and of every later one are awaited directly)
      const uint32_t first = it > (uint32_t)a.ns ? it - (uint32_t)a.ns : 0u;
      bool ab = *abort_flag != 0;
      for (uint32_t k = first; k < it; k++) {
        const int s = (int)(k % (uint32_t)a.ns);
        const uint32_t ph = (k / (uint32_t)a.ns) & 1u;
        if (!ab && ptx::mbar_wait(EMPTY + 8u * s, ph, abort_flag, TC_WAIT_NS)) continue;
        ab = true;
        ptx::mbar_wait(FULL + 8u * s, ph, nullptr, TC_WAIT_NS / 8);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      uint32_t it = 0;
      const int ksteps = a.kpad / 16;
      // the forced wait can only run out: it raises the abort flag and no MMA is issued
      const bool go = a.forced_wait_ns == 0 || ptx::mbar_wait(NEVER, 0u, abort_flag, a.forced_wait_ns);
      for (int q = 0; go && q < nq; q++) {
        const int ab = q & 1;
        const uint32_t aph = ((uint32_t)q >> 1) & 1u;
        if (!ptx::mbar_wait(ACCE + 8u * ab, aph ^ 1u, abort_flag, TC_WAIT_NS)) break;
        ptx::tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(ab * a.nmma);
        bool ok = true;
        for (int t = 0; t < ni; t++) {
          const int s = (int)(it % (uint32_t)a.ns);
          const uint32_t ph = (it / (uint32_t)a.ns) & 1u;
          if (!ptx::mbar_wait(FULL + 8u * s, ph, abort_flag, TC_WAIT_NS)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t as = sA + (uint32_t)(s * a.a_bytes), bs = sB + (uint32_t)(s * a.bslot);
          for (int kk = 0; kk < ksteps; kk++)
            ptx::mma_f16(dt, ptx::smem_desc(as + 256u * kk, 128u, (uint32_t)a.sbo),
                         ptx::smem_desc(bs + 256u * kk, 128u, (uint32_t)a.sbo), a.idesc, (t | kk) != 0);
          ptx::mma_commit(EMPTY + 8u * s);
          it++;
        }
        if (!ok) break;
        ptx::mma_commit(ACCF + 8u * ab);
      }
      // every MMA of this CTA has completed before tensor memory is released
      ptx::mma_commit(FIN);
      ptx::mbar_wait(FIN, 0u, nullptr, TC_WAIT_NS);
    }
    __syncwarp();
  } else {
    // ---- epilogue: accumulator rows -> y ----
    const int sub = warp & 3;            // lane quarter of tensor memory this warp may read
    const int row = sub * 32 + lane;     // accumulator row 2 i + c
    const int i = row >> 1, c = row & 1;
    const int rh = (a.Rk + 1) / 2, rlo = c ? rh : 0, rhi = c ? a.Rk : rh;
    const bool pad_row = i >= a.n && i < a.kpad;
    const bool last_chunk = a.r0 + a.Rk == a.R;
    for (int q = 0; q < nq; q++) {
      const int idx = (int)blockIdx.x + q * G;
      const int ab = q & 1;
      const uint32_t aph = ((uint32_t)q >> 1) & 1u;
      int ok = 0;
      if (lane == 0) ok = ptx::mbar_wait(ACCF + 8u * ab, aph, abort_flag, TC_WAIT_NS) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      ptx::tc_fence_after();
      uint32_t raw[NGJ * 8];
      const uint32_t tbase = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(ab * a.nmma);
#pragma unroll
      for (int g = 0; g < NGJ; g++) ptx::tmem_ld8(tbase + 8u * g, raw + 8 * g);
      ptx::tmem_wait_ld();
      float dv[NGJ * 8];
#pragma unroll
      for (int j = 0; j < NGJ * 8; j++) dv[j] = ptx::tmem_reg(raw[j]);
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ACCE + 8u * ab);

      char* img = a.yt ? a.yt + (size_t)idx * a.b_bytes : nullptr;
#pragma unroll
      for (int rr = 0; rr < NGJ * 4; rr++) {
        const float oa = dv[2 * rr], ob = dv[2 * rr + 1];
        const float pa = __shfl_xor_sync(0xffffffffu, oa, 1), pb = __shfl_xor_sync(0xffffffffu, ob, 1);
        if (rr < rlo || rr >= rhi) continue;
        const int r = a.r0 + rr;
        if (i < a.n) {
          float re = (c ? pa - ob : oa - pb) * a.sres;
          float im = (c ? pb + oa : ob + pa) * a.sres;
          const size_t o = ((size_t)idx * a.n + i) * a.R + r;
          if (a.xs) {
            const float2 xv = a.xs_half ? ld_f2((const __half2*)a.xs, o) : ld_f2((const float2*)a.xs, o);
            const float m = (i < a.nv ? a.mu_c : -a.mu_c) * a.sres;
            re -= m * xv.y;
            im += m * xv.x;
          }
          if (a.sy != 0.f) {
            const float2 yv = a.yin[o];
            re += a.sy * yv.x;
            im += a.sy * yv.y;
          }
          if (a.y) a.y[o] = make_float2(re, im);
          if (img) {
            *reinterpret_cast<__half*>(img + img_off(2 * r, i, a.sbo)) = __float2half_rn(re);
            *reinterpret_cast<__half*>(img + img_off(2 * r + 1, i, a.sbo)) = __float2half_rn(im);
          }
        } else if (img && pad_row) {
          *reinterpret_cast<__half*>(img + img_off(2 * r, i, a.sbo)) = __float2half_rn(0.f);
          *reinterpret_cast<__half*>(img + img_off(2 * r + 1, i, a.sbo)) = __float2half_rn(0.f);
        }
      }
      // columns of the last 8-wide group beyond 2R are zero in the image
      if (img && last_chunk && c == 0 && i < a.kpad)
        for (int j = 2 * a.R; j < 8 * a.ngj_all; j++)
          *reinterpret_cast<__half*>(img + img_off(j, i, a.sbo)) = __float2half_rn(0.f);
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, 1);
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, (uint32_t)a.tcols);
  }
}

// ---- host side -------------------------------------------------------------------------------
static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

size_t tc_vector_image_bytes(const CoarseLevel& c, int nsites, int R) {
  return (size_t)nsites * tc_geom(c.n, R).b_bytes;
}

void launch_vector_image(const CoarseLevel& c, void* img, const void* x, int x_type, int nsites, int R, cudaStream_t st) {
  TcGeom t = tc_geom(c.n, R);
  ScopedTimer timer_("coarse_image", st, R,
                     (double)nsites * ((double)c.n * R * (x_type == 2 ? 4 : 8) + t.b_bytes));
  size_t tot = (size_t)nsites * 8 * t.ngj * (t.kpad / 8);
  if (!tot) return;
  const unsigned grid = (unsigned)((tot + 255) / 256);
  if (x_type == 2)
    k_vector_image<__half2><<<grid, 256, 0, st>>>((char*)img, (const __half2*)x, nsites, c.n, R, t.kpad, t.sbo, t.ngj,
                                                  t.b_bytes);
  else if (x_type == 1)
    k_vector_image<float2><<<grid, 256, 0, st>>>((char*)img, (const float2*)x, nsites, c.n, R, t.kpad, t.sbo, t.ngj,
                                                 t.b_bytes);
  else
    throw Error(DDTM_ERR_ARG, "internal: vector image input type");
  CKL("vector_image");
}

static void matrix_images(const CoarseLevel& c, char* img, const float2* src, size_t nblocks, cudaStream_t st) {
  TcGeom t = tc_geom(c.n, 1);
  size_t tot = nblocks * t.arows * (t.kpad / 8);
  if (!tot) return;
  k_matrix_image<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(img, src, nblocks, c.n, t.arows, t.kpad, t.sbo,
                                                                t.a_bytes);
  CKL("matrix_image");
}

void build_coarse_images(CoarseLevel& c, cudaStream_t st) {
  if (!tc_supported(c.n)) throw Error(DDTM_ERR_ARG, "tensor-core coarse operator needs 2 n_v <= 64");
  TcGeom t = tc_geom(c.n, 1);
  c.Dct.ensure((size_t)c.Nc * 9 * t.a_bytes);
  matrix_images(c, c.Dct.as<char>(), c.Dc.as<float2>(), (size_t)c.Nc * 9, st);
  c.tc_err.ensure(sizeof(int));
  CK(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), st));
}


// Images of B = Dinv(e) A_d(e), d = 1..8, for every even site e: thread (block, row pair i, column group
// h) forms B[i][8h .. 8h+7] (FP32 sums over k in order) and writes image rows 2i (real parts) and 2i + 1
// (imaginary parts); rows and columns beyond n are the zero padding.  Both factors are column-major
// n x n blocks.
__global__ void k_hop_inverse_image(char* __restrict__ img, const float2* __restrict__ Dinv,
                                    const float2* __restrict__ Dc, const int* __restrict__ even, int ne, int n,
                                    int arows, int kpad, int sbo, int a_bytes) {
  const int kg = kpad / 8, hrows = arows / 2;
  const size_t per = (size_t)hrows * kg;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)ne * 8 * per) return;
  const size_t b = tid / per;  // block e * 8 + (d - 1)
  const int rem = (int)(tid - b * per), i = rem % hrows, h = rem / hrows;
  const int e = (int)(b / 8), d = (int)(b % 8) + 1;
  const float2* Di = Dinv + (size_t)e * n * n;                       // column k at Di + k n
  const float2* Ad = Dc + ((size_t)__ldg(even + e) * 9 + d) * n * n;  // column j at Ad + j n
  float re[8], im[8];
#pragma unroll
  for (int q = 0; q < 8; q++) re[q] = im[q] = 0.f;
  if (i < n) {
    for (int k = 0; k < n; k++) {
      const float2 a = __ldg(Di + (size_t)k * n + i);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int j = 8 * h + q;
        if (j < n) {
          const float2 bkj = __ldg(Ad + (size_t)j * n + k);
          re[q] += a.x * bkj.x - a.y * bkj.y;
          im[q] += a.x * bkj.y + a.y * bkj.x;
        }
      }
    }
  }
  __align__(16) __half vr[8], vi[8];
#pragma unroll
  for (int q = 0; q < 8; q++) {
    vr[q] = __float2half_rn(re[q]);
    vi[q] = __float2half_rn(im[q]);
  }
  char* base = img + b * a_bytes;
  *reinterpret_cast<uint4*>(base + img_off(2 * i, 8 * h, sbo)) = *reinterpret_cast<const uint4*>(vr);
  *reinterpret_cast<uint4*>(base + img_off(2 * i + 1, 8 * h, sbo)) = *reinterpret_cast<const uint4*>(vi);
}

void build_inverse_images(CoarseLevel& c, cudaStream_t st) {
  TcGeom t = tc_geom(c.n, 1);
  const size_t ne = c.h_even.size();
  c.Dhopt.ensure(ne * 8 * t.a_bytes);
  const size_t tot = ne * 8 * (size_t)(t.arows / 2) * (t.kpad / 8);
  if (!tot) return;
  k_hop_inverse_image<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c.Dhopt.as<char>(), c.Dinv.as<float2>(),
                                                                     c.Dc.as<float2>(), c.even.as<int>(), (int)ne,
                                                                     c.n, t.arows, t.kpad, t.sbo, t.a_bytes);
  CKL("hop_inverse_image");
}

// ---- autotuner ---------------------------------------------------------------------------------
// Per pass shape (column groups, rows, outputs, operands) the first launch outside stream capture
// times every admissible residency (1, 2 or 3 CTAs per SM; the ring of stages fills the shared memory
// left per CTA) and keeps the fastest.  A pass computes each output from the same MMAs in the same
// order whatever the residency, so the choice changes the time, never the result; only passes that
// overwrite their outputs (no accumulation into y) are re-run for timing.
namespace {
struct TcTune {
  std::mutex m;
  std::map<std::string, int> cps;                    // shape -> CTAs per SM
  std::map<std::string, std::vector<float>> ms;     // shape -> time of each candidate (index = cps - 1)
  bool on = true;
};
TcTune& tune() {
  static TcTune t;
  return t;
}
}  // namespace

void tc_autotune_enable(bool on) { tune().on = on; }

void tc_set_forced_wait_ns(uint64_t ns) { g_forced_wait_ns.store(ns); }
uint64_t tc_forced_wait_ns() { return g_forced_wait_ns.load(); }

std::string tc_autotune_report() {
  TcTune& t = tune();
  std::lock_guard<std::mutex> lock(t.m);
  std::string out = "{";
  bool first = true;
  for (auto& kv : t.cps) {
    char buf[256];
    std::string times;
    for (float v : t.ms[kv.first]) {
      char b2[32];
      snprintf(b2, sizeof(b2), "%s%.4f", times.empty() ? "" : ", ", v);
      times += b2;
    }
    snprintf(buf, sizeof(buf), "%s\"%s\": {\"ctas_per_sm\": %d, \"ms\": [%s]}", first ? "" : ", ", kv.first.c_str(),
             kv.second, times.c_str());
    out += buf;
    first = false;
  }
  return out + "}";
}

static void launch_coarse_tc_cps(const CoarseLevel& c, const TcPass& p, int R, cudaStream_t st, int cps_force);

void launch_coarse_tc(const CoarseLevel& c, const TcPass& p, int R, cudaStream_t st) {
  TcTune& t = tune();
  const int ngj = (2 * (R < 32 ? R : 32) + 7) / 8;
  char key[160];
  snprintf(key, sizeof(key), "%s|n%d|R%d|out%d|s%d|h%d", p.name, c.n, R, p.nout, (int)p.self, (int)p.hops);
  int chosen = 0;
  {
    std::lock_guard<std::mutex> lock(t.m);
    auto it = t.cps.find(key);
    if (it != t.cps.end()) chosen = it->second;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  const bool idempotent = !(p.y && p.yin && p.sy != 0.f);
  if (chosen || !t.on || cap != cudaStreamCaptureStatusNone || !idempotent || p.nout <= 0 || timer_on() ||
      g_forced_wait_ns.load()) {
    launch_coarse_tc_cps(c, p, R, st, chosen);
    return;
  }
  // candidates: every residency the registers allow (ngj <= 4: up to 2 per SM; ngj <= 2: 3)
  const int maxc = ngj <= 2 ? 3 : tc_ctas_per_sm(ngj);
  std::vector<float> ms(maxc, 0.f);
  cudaEvent_t ev[2];
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  int best = 1;
  for (int cand = 1; cand <= maxc; cand++) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
      CK(cudaEventRecord(ev[0], st));
      launch_coarse_tc_cps(c, p, R, st, cand);
      CK(cudaEventRecord(ev[1], st));
      CK(cudaEventSynchronize(ev[1]));
      float v = 0;
      CK(cudaEventElapsedTime(&v, ev[0], ev[1]));
      if (rep > 0 && v < tmin) tmin = v;  // the first run warms caches and the module
    }
    ms[cand - 1] = tmin;
    if (tmin < ms[best - 1]) best = cand;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  {
    std::lock_guard<std::mutex> lock(t.m);
    t.cps[key] = best;
    t.ms[key] = ms;
  }
  launch_coarse_tc_cps(c, p, R, st, best);  // the launch the caller asked for
}

static void launch_coarse_tc_cps(const CoarseLevel& c, const TcPass& p, int R, cudaStream_t st, int cps_force) {
  TcGeom t = tc_geom(c.n, R);
  // algorithmic bytes: the matrix images, each input vector image once, the outputs
  double bytes = (double)p.nout * ((p.self ? 1 : 0) + (p.hops ? 8 : 0)) * t.a_bytes;
  bytes += (double)p.nout * t.b_bytes * ((p.self ? 1 : 0) + (p.hops && p.X_hop != p.X_self ? 1 : 0));
  if (p.y) bytes += (double)p.nout * c.n * R * 8;
  if (p.yt) bytes += (double)p.nout * t.b_bytes;
  if (p.xs) bytes += (double)p.nout * c.n * R * (p.xs_type == 2 ? 4 : 8);
  ScopedTimer timer_(p.name, st, R, bytes);
  if (p.nout <= 0) return;
  for (int r0 = 0; r0 < R; r0 += 32) {
    const int Rk = R - r0 < 32 ? R - r0 : 32;
    const int ngj = (2 * Rk + 7) / 8, nmma = (2 * Rk + 15) / 16 * 16 < 16 ? 16 : (2 * Rk + 15) / 16 * 16;
    TcArgs a;
    a.A_self = (const char*)p.A_self;
    a.a_self_stride = p.a_self_stride;
    a.self_by_site = p.self_by_site;
    a.A_hop = (const char*)p.A_hop;
    a.hop_by_slot = p.hop_by_slot ? 1 : 0;
    a.X_self = (const char*)p.X_self;
    a.X_hop = (const char*)p.X_hop;
    a.tab = p.tab;
    a.osite = p.osite;
    a.nout = p.nout;
    a.self = p.self ? 1 : 0;
    a.hops = p.hops ? 1 : 0;
    a.y = reinterpret_cast<float2*>(p.y);
    a.yin = reinterpret_cast<const float2*>(p.yin);
    a.xs = p.xs;
    if (p.xs && p.xs_type != 1 && p.xs_type != 2) throw Error(DDTM_ERR_ARG, "internal: twist vector type");
    a.xs_half = p.xs_type == 2;
    a.sy = p.sy;
    a.sres = p.sres;
    a.mu_c = p.mu_c;
    a.yt = (char*)p.yt;
    a.n = c.n;
    a.nv = c.nv;
    a.R = R;
    a.r0 = r0;
    a.Rk = Rk;
    a.kpad = t.kpad;
    a.sbo = t.sbo;
    a.a_bytes = t.a_bytes;
    a.b_bytes = t.b_bytes;
    a.ngj_all = t.ngj;
    a.nmma = nmma;
    a.bslot = nmma / 8 * t.sbo;
    a.apad = (128 - t.arows) / 8 * t.sbo;
    const int cps = cps_force > 0 ? cps_force : tc_ctas_per_sm(ngj), budget = tc_smem_budget(cps);
    a.ns = (budget - a.apad) / (a.a_bytes + a.bslot);
    if (a.ns > TC_MAXNS) a.ns = TC_MAXNS;
    if (a.ns < 2) throw Error(DDTM_ERR_ARG, "tensor-core coarse stencil: blocks too large for the stage ring");
    int tc = 32;
    while (tc < 2 * nmma) tc *= 2;
    a.tcols = tc;
    a.idesc = ptx::idesc_f16_f32(128, nmma);
    a.err = c.tc_err.as<int>();
    a.forced_wait_ns = g_forced_wait_ns.load();
    const size_t smem = (size_t)a.ns * (a.a_bytes + a.bslot) + a.apad + 1024;
    const int grid = p.nout < cps * num_sms() ? p.nout : cps * num_sms();
#define TC_LAUNCH(K)                                                                                    \
  case K: {                                                                                           \
    set_dynamic_smem((const void*)k_coarse_tc<K>, TC_SMEM_1 + 1024);                                  \
    k_coarse_tc<K><<<grid, 192, smem, st>>>(a);                                                       \
    break;                                                                                            \
  }
    switch (ngj) {
      TC_LAUNCH(1)
      TC_LAUNCH(2)
      TC_LAUNCH(3)
      TC_LAUNCH(4)
      TC_LAUNCH(5)
      TC_LAUNCH(6)
      TC_LAUNCH(7)
      TC_LAUNCH(8)
      default:
        throw Error(DDTM_ERR_ARG, "internal: column groups");
    }
#undef TC_LAUNCH
    CKL("coarse_tc");
  }
}

void check_tc_error(CoarseLevel& c) {
  if (!c.tc_err.p) return;
  int e = 0;
  CK(cudaMemcpy(&e, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(cudaMemset(c.tc_err.p, 0, sizeof(int)));
    throw Error(DDTM_ERR_TIMEOUT, "tensor-core coarse stencil: a pipeline wait timed out");
  }
}

}  // namespace ddtm

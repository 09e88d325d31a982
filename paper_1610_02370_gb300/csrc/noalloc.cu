// ddtm_apply_D_noalloc: y = D(mu) x for callers that must not allocate device
// memory during the call.  cudaMalloc and cudaFree may synchronise the whole
// device and stall every stream, and some applications hand the whole memory
// budget of the GPU to their own allocator up front; both kinds of caller need
// an operator application that takes its working memory from somewhere fixed.
//
// The canonical-layout apply needs two fields in the internal even-odd block
// layout (the converted x and the result before conversion back).  Here they
// live in one file-scope device array of fixed size, shared by every call on a
// device and kept by the GPU that loaded the library until the process exits.
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "ddtm_internal.h"
#include "solver.h"

using namespace ddtm;

// 64 MiB: two FP64 fields of up to 174762 sites (e.g. 16^3 x 32 = 131072)
#define NOALLOC_SCRATCH_BYTES (64u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the array, looked up once per device with that device
// current (in host code the symbol's name is only a host-side stand-in).  The
// per-device cache is guarded by a mutex, so host threads making their first
// call at the same time do not race on it.
static void* scratch_address(int dev) {
  static std::mutex mtx;
  static void* addr[128] = {nullptr};
  if (dev < 0 || dev >= 128) throw Error(DDTM_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(mtx);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw Error(DDTM_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                     cudaGetErrorString(e));
    }
    addr[dev] = p;
  }
  return addr[dev];
}

// Device (or managed) memory of device dev; otherwise an error naming what was found.
static void require_device_pointer(const void* p, int dev, const char* name) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    throw Error(DDTM_ERR_ARG, std::string(name) + " is not a CUDA pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    throw Error(DDTM_ERR_ARG, std::string(name) + " is not device memory (host or unregistered pointer)");
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    throw Error(DDTM_ERR_ARG, std::string(name) + " is memory of device " + std::to_string(a.device) +
                                  ", the current device is " + std::to_string(dev));
}

extern "C" int ddtm_apply_D_noalloc(ddtm_ctx* ctx, double* y, const double* x, double mu, int prec) {
  if (!ctx) return DDTM_ERR_ARG;
  ctx->err.clear();
  try {
    check_prec(prec);
    if (!x || !y || x == y) throw Error(DDTM_ERR_ARG, "x and y must be distinct device pointers");
    const FineGeom& g = ctx->g;
    size_t s2 = store2_bytes(prec);
    size_t field = (size_t)g.V * 12 * s2;
    size_t nrm = prec == PREC_F16 ? (size_t)g.V * sizeof(float) : 0;
    size_t field_al = (field + 255) / 256 * 256, nrm_al = (nrm + 255) / 256 * 256;
    size_t need = 2 * (field_al + nrm_al);
    if (need > NOALLOC_SCRATCH_BYTES)
      throw Error(DDTM_ERR_ARG, "lattice of " + std::to_string(g.V) + " sites needs " + std::to_string(need) +
                                    " bytes of scratch in this precision; the fixed array holds " +
                                    std::to_string((size_t)NOALLOC_SCRATCH_BYTES));
    require_gauge(ctx);
    if (!ctx->links[prec].p || !ctx->clover[prec].p)
      throw Error(DDTM_ERR_STATE, "gauge field not yet held in this precision (one ddtm_apply_D call with it "
                                  "creates that copy); FP64 is always present");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    require_device_pointer(x, dev, "x");
    require_device_pointer(y, dev, "y");
    char* base = (char*)scratch_address(dev);
    void* xi = base;
    float* xin = prec == PREC_F16 ? (float*)(base + field_al) : nullptr;
    void* yi = base + field_al + nrm_al;
    float* yin = prec == PREC_F16 ? (float*)(base + 2 * field_al + nrm_al) : nullptr;
    launch_spinor_from_canon(g, prec, xi, xin, x, ctx->stream);
    launch_dslash(g, prec, yi, yin, xi, xin, ctx->links[prec].p, ctx->clover[prec].p, mu, ctx->stream);
    launch_spinor_to_canon(g, prec, yi, yin, y, ctx->stream);
  } catch (const Error& e) {
    ctx->err = e.what();
    return e.code;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return DDTM_ERR_CUDA;
  }
  return DDTM_OK;
}

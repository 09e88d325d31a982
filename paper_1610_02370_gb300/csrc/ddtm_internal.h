// Host-side internals of libddtm: the context, device buffers, geometry and
// the launch wrappers that the C ABI (api.cu) and the solvers call.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ddtm.h"

namespace ddtm {

// Error carrying a DDTM_ERR_* code; thrown inside the library, turned into a
// return status at the C boundary.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void cuda_check(cudaError_t e, const char* what);
// after every kernel launch: counts the launch (kernel_launches()) and checks it
void cuda_check_launch(const char* what);
long kernel_launches();
// kernels launched by a graph replay count like direct launches
void add_kernel_launches(long n);
#define CK(x) ::ddtm::cuda_check((x), #x)
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute belongs to a (kernel, device) pair, so the
// limits already set are remembered per pair; safe to call from several host
// threads.
void set_dynamic_smem(const void* kernel, size_t bytes);
#define CKL(what) ::ddtm::cuda_check_launch(what)

// Device bytes held by the library's allocations (every DevBuf of the
// process) and the optional cap on them (0: none); an allocation beyond the
// cap throws DDTM_ERR_OOM without calling cudaMalloc.
size_t device_bytes_in_use();
void set_device_memory_limit(size_t bytes);
size_t device_memory_limit();
// changes whenever any library device buffer is allocated or freed (a cached
// CUDA graph is valid only within one generation: its kernels hold pointers)
long alloc_generation();

// Owned device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() {}
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release();
  void ensure(size_t n);  // grow to at least n bytes (contents not kept)
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Fine-lattice geometry in the internal block layout (see common.cuh).
struct FineGeom {
  int L[4];   // lattice extent per direction mu = t, x, y, z
  int b[4];   // block extent per direction
  int NB[4];  // blocks per direction
  int Vb = 0, Nb = 0;
  long V = 0;
  int bc_t = 0;
  std::vector<uint32_t> h_loc_nbr, h_loc_coord;
  std::vector<int> h_blk_nbr;
  DevBuf loc_nbr, loc_coord, blk_nbr;
  DevBuf colour_blocks;  // [2][Nb/2]: blocks of colour 0 (red), then colour 1 (black)
};

// One coarse level: a lattice of aggregates with 2*nv dofs per site.
struct CoarseLevel {
  int lat[4];        // extent per direction mu
  int Nc = 0;        // sites
  int nv = 0, n = 0; // n = 2 nv
  std::vector<int> h_nbr;      // [8][Nc] neighbour site, hop k = 2 mu + (0 fwd, 1 bwd)
  std::vector<int> h_even, h_odd;
  // parity-compact neighbour tables: [8][No] even-list index of the neighbour
  // of odd site i, and [8][Ne] odd-list index of the neighbour of even site i
  std::vector<int> h_nbr_oe, h_nbr_eo;
  DevBuf nbr, even, odd, nbr_oe, nbr_eo;  // device copies
  int prec = 1;                // F32: SIMT stencil; F16: tensor-core stencil on FP16 images
  DevBuf Dc;                   // [site][9][col][row] complex FP32, see coarse.cu
  DevBuf Dinv;                 // inverses of (self + i mu_c Gamma5_c) on even sites, FP32
  DevBuf Dct;                  // FP16 matrix images of Dc (prec F16), see coarse_tc.cu
  DevBuf Dhopt;                // FP16 images of Dinv(e) A_d(e), the 8 hops of every even site (prec F16)
  DevBuf tc_err;               // set by a tensor-core pass that gave up waiting
  double inv_mu = 0;
  bool inv_valid = false;
  bool built = false;
};

// Aggregation of the level-1 lattice (three-level hierarchies, Sec. 2.3 applied
// to D_1): aggregates are blocks of b[4] level-1 sites (also the blocks of the
// level-1 SAP smoother, Sec. 2.4); they are the sites of level 2, in canonical
// order over the NB[4] block lattice.  Within an aggregate the sites are
// numbered q in canonical order of their offsets.
struct Level1Agg {
  int b[4] = {0, 0, 0, 0}, NB[4] = {0, 0, 0, 0};
  int Nagg = 0, Vb = 0;
  int nv = 0;                 // level-1 test vectors (columns of P_1 per aggregate half)
  std::vector<int> h_sites;   // [Nagg][Vb] level-1 site of local index q
  DevBuf sites;               // device copy of h_sites
  DevBuf colour;              // [2][Nagg/2]: aggregates of colour 0 (red), then colour 1
  DevBuf tabs;                // [9][8][Nc1 + 1] neighbour tables of the Galerkin parts (see level1.cu)
  DevBuf tv;                  // [nv][Nc1][n1] level-1 test vectors, complex FP32
  DevBuf P;                   // [Nagg][2][nv][Vb][n1/2] P_1, complex FP32
  bool geom = false;
};

// faces of a block: for hop k, the sites whose hop leaves the block
struct FaceDev {
  DevBuf idx, list;
  int off[9] = {0};
};

// Pinned host ring of coefficient blocks copied to the device asynchronously;
// each slot carries an event so a slot is reused only after its copy is done.
struct CoefRing {
  static const int SLOTS = 64;
  size_t slot_elems = 0;
  double2* host = nullptr;
  DevBuf dev;
  cudaEvent_t ev[SLOTS];
  bool ev_used[SLOTS] = {false};
  int next = 0;
  CoefRing() {}
  CoefRing(const CoefRing&) = delete;
  CoefRing& operator=(const CoefRing&) = delete;
  ~CoefRing();
  // copy count values to a device slot (asynchronously on st) and return it
  const double2* push(const double2* vals, size_t count, cudaStream_t st);
};

struct ScratchPool {
  std::map<std::string, DevBuf*> bufs;
  ~ScratchPool();
  void* get(const std::string& name, size_t bytes);
  void clear();                                       // frees every buffer
  size_t held(const std::string& prefix) const;  // bytes held by buffers whose name starts with prefix
};

}  // namespace ddtm

struct ddtm_field {
  ddtm_ctx* ctx;
  int prec;
  int nrhs;
  size_t stride;  // complex elements per rhs (12 * V)
  ddtm::DevBuf data;
  ddtm::DevBuf nrm;  // FP16 only: one float per site and rhs
};

struct ddtm_ctx {
  ddtm::FineGeom g;
  cudaStream_t stream = 0;
  std::string err;
  ddtm_params p;
  bool gauge = false;
  double kappa = 0, csw = 0;
  double theta[4] = {0, 0, 0, 0};  // twisted boundary phases applied to the internal links
  ddtm::DevBuf links[3];   // per precision, internal layout
  ddtm::DevBuf clover[3];  // per precision, packed site term (incl. m+4)
  ddtm::DevBuf sinv[3];    // per precision, even-site inverse of site term + i mu gamma5
  double sinv_mu[3] = {0, 0, 0};
  bool sinv_ok[3] = {false, false, false};
  // level-0 aggregation
  int nv0 = 0;
  ddtm::DevBuf tv0;        // test vectors: nv0 fine FP32 fields (internal layout)
  ddtm::DevBuf P0;         // orthonormalised P, FP32: [blk][s][i][6][Vb] complex
  ddtm::DevBuf P0h;        // FP16 copy of P0
  ddtm::FaceDev faces;
  bool faces_ready = false;
  ddtm::CoarseLevel c1;
  bool c1_geom = false;
  // three levels: aggregation of level 1 and the coarsest operator D_2
  ddtm::Level1Agg a1;
  ddtm::CoarseLevel c2;
  bool c2_geom = false;
  long coarse_iters = 0;   // accumulated by the coarsest solves
  ddtm::CoefRing ring;     // coefficient transfers of the Krylov solvers
  bool have_P = false;
  bool setup_done = false;
  double setup_mu = 0;
  double setup_s = 0;
  ddtm::ScratchPool scratch;
  // pinned host scratch and named event pairs (created on first use, kept)
  std::map<std::string, std::pair<void*, size_t>> host_bufs;
  std::map<std::string, std::pair<cudaEvent_t, cudaEvent_t>> event_pairs;
  // CUDA graphs of repeated launch sequences (one coarsest-GMRES iteration),
  // keyed by everything their kernels' arguments depend on; value: the
  // executable graph and its number of kernel nodes
  std::map<std::string, std::pair<cudaGraphExec_t, int>> graphs;
  bool use_graphs = true;   // option "graphs"
  long graphs_gen = -1;     // allocation generation the cached graphs belong to
  cudaStream_t capture_stream = nullptr;  // private stream that graphs are captured on
  void* scratch_host(const std::string& name, size_t bytes);
  void events(const std::string& name, cudaEvent_t ev[2]);
  ~ddtm_ctx();
};

namespace ddtm {

// ---- geometry.cu -------------------------------------------------------------
void build_geometry(FineGeom& g);
void build_coarse_geometry(const FineGeom& g, CoarseLevel& c);
// neighbour tables and parity lists of a coarse lattice with extents lat[4] (mu order)
void build_coarse_geometry_lat(const int lat[4], CoarseLevel& c);
// aggregates of b[4] sites on the level-1 lattice of c1
void build_level1_aggregates(const CoarseLevel& c1, const int b[4], Level1Agg& a);
// canonical FP64 complex spinor (one rhs) <-> internal field of precision prec
void launch_spinor_from_canon(const FineGeom& g, int prec, void* d, float* nrm, const double* in, cudaStream_t s);
void launch_spinor_to_canon(const FineGeom& g, int prec, const void* d, const float* nrm, double* out, cudaStream_t s);
// canonical FP64 links -> internal FP64 links
void launch_links_from_canon(const FineGeom& g, double* out, const double* U, cudaStream_t s);
// element-wise precision conversion of complex arrays (double2 -> float2 / half2)
void launch_convert_complex(const double* in, int prec_out, void* out, size_t n, cudaStream_t s);
// U_mu(x) *= exp(i phase[mu]) on the sites with x_mu = L_mu - 1 (internal FP64 links)
void launch_link_phases(const FineGeom& g, double* links, const double phase[4], cudaStream_t s);
// count non-finite doubles
void launch_count_nonfinite(const double* a, size_t n, int* counter, cudaStream_t s);

// ---- dirac.cu --------------------------------------------------------------------
void launch_clover_build(const FineGeom& g, double* clov, const double* Ucanon, double m_plus_4, double csw,
                         cudaStream_t s);
void launch_site_inverse(const FineGeom& g, int prec, void* out, const double* clov64, double mu, cudaStream_t s);
void launch_dslash(const FineGeom& g, int prec, void* y, float* ynrm, const void* x, const float* xnrm,
                   const void* links, const void* clover, double mu, cudaStream_t s);
// nrhs right-hand sides at stride 12 V (FP16 scales at stride V), one launch where the block kernel applies
void launch_dslash_multi(const FineGeom& g, int prec, void* y, float* ynrm, const void* x, const float* xnrm,
                         const void* links, const void* clover, double mu, int nrhs, cudaStream_t s);

// ---- sap.cu ----------------------------------------------------------------------
void launch_sap_half(const FineGeom& g, int prec, void* x, float* xn, const void* b, const float* bn, const void* links,
                     const void* clover, const void* sinv, const int* blocks, const int* zero_blocks, int nblocks,
                     int zero_x, int nmr, double mu, int nrhs, cudaStream_t s);

}  // namespace ddtm

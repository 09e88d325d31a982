// Lattice geometry of the internal even-odd block layout, the tables the
// stencil kernels use to find neighbours, and the kernels that convert between
// the canonical FP64 layout of the C ABI and the internal layout.
//
// Internal site s = blk * Vb + loc with blk the canonical index of the block
// over the block lattice and loc = parity * Vb/2 + (lexloc >> 1).  Because every
// block extent is even, block origins have even parity, so the local parity is
// the global parity (t + x + y + z) mod 2, and each x-row of a block holds
// alternating parities, which makes (parity, lexloc >> 1) a bijection.
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "ddtm_internal.h"
#include "timer.h"

namespace ddtm {

static std::atomic<long> g_kernel_launches{0};
long kernel_launches() { return g_kernel_launches.load(); }
void add_kernel_launches(long n) { g_kernel_launches.fetch_add(n); }
void cuda_check_launch(const char* what) {
  g_kernel_launches.fetch_add(1);
  cuda_check(cudaGetLastError(), what);
}

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    int code = (e == cudaErrorMemoryAllocation) ? DDTM_ERR_OOM : DDTM_ERR_CUDA;
    throw Error(code, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void set_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex m;
  static std::map<std::pair<const void*, int>, size_t> set;  // (kernel, device) -> limit set
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(m);
  size_t& have = set[std::make_pair(kernel, dev)];
  if (bytes <= have) return;
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
}

// Device bytes held by every DevBuf of the process, and the caller's budget
// for them (0: none).
static std::atomic<size_t> g_dev_bytes{0};
static std::atomic<long> g_alloc_gen{0};  // bumped by every device allocation and free of a DevBuf
long alloc_generation() { return g_alloc_gen.load(); }
static std::atomic<size_t> g_dev_limit{0};
size_t device_bytes_in_use() { return g_dev_bytes.load(); }
void set_device_memory_limit(size_t bytes) { g_dev_limit.store(bytes); }
size_t device_memory_limit() { return g_dev_limit.load(); }

void DevBuf::release() {
  if (p) {
    cudaFree(p);
    g_dev_bytes.fetch_sub(bytes);
    g_alloc_gen.fetch_add(1);
  }
  p = nullptr;
  bytes = 0;
}

void DevBuf::ensure(size_t n) {
  if (n <= bytes && p) return;
  release();
  if (n == 0) return;
  const size_t lim = g_dev_limit.load();
  if (lim && g_dev_bytes.load() + n > lim)
    throw Error(DDTM_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes would exceed the library's "
                                  "memory limit of " + std::to_string(lim) + " bytes (" +
                                  std::to_string(g_dev_bytes.load()) + " in use)");
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    throw Error(DDTM_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed");
  }
  bytes = n;
  g_dev_bytes.fetch_add(n);
  g_alloc_gen.fetch_add(1);
}

ScratchPool::~ScratchPool() { clear(); }

void ScratchPool::clear() {
  for (auto& kv : bufs) delete kv.second;
  bufs.clear();
}

void* ScratchPool::get(const std::string& name, size_t bytes) {
  auto it = bufs.find(name);
  DevBuf* b;
  if (it == bufs.end()) {
    b = new DevBuf();
    bufs[name] = b;
  } else {
    b = it->second;
  }
  b->ensure(bytes < 256 ? 256 : bytes);
  return b->p;
}

size_t ScratchPool::held(const std::string& prefix) const {
  size_t s = 0;
  for (const auto& kv : bufs)
    if (kv.first.compare(0, prefix.size(), prefix) == 0) s += kv.second->bytes;
  return s;
}

// local coordinates (per direction t, x, y, z) of local index loc
static void loc_coords(const int b[4], int loc, int c[4]) {
  int Vh = b[0] * b[1] * b[2] * b[3] / 2;
  int par = loc / Vh;
  int h = loc % Vh;
  int two_h = 2 * h;
  int bx = b[1], by = b[2], bz = b[3];
  int xe = two_h % bx;  // even x offset of the pair
  int r = two_h / bx;
  int ly = r % by;
  r /= by;
  int lz = r % bz;
  int lt = r / bz;
  int lx = xe + ((par + lt + lz + ly) & 1);
  c[0] = lt; c[1] = lx; c[2] = ly; c[3] = lz;
}

static int loc_index(const int b[4], const int c[4]) {
  int lex = ((c[0] * b[3] + c[3]) * b[2] + c[2]) * b[1] + c[1];
  int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  return par * (b[0] * b[1] * b[2] * b[3] / 2) + (lex >> 1);
}

// canonical order over a lattice with per-direction extents n[4]: x fastest, then y, z, t
static int canon_index(const int n[4], const int c[4]) {
  return ((c[0] * n[3] + c[3]) * n[2] + c[2]) * n[1] + c[1];
}
static void canon_coords(const int n[4], int i, int c[4]) {
  c[1] = i % n[1]; i /= n[1];
  c[2] = i % n[2]; i /= n[2];
  c[3] = i % n[3];
  c[0] = i / n[3];
}

void build_geometry(FineGeom& g) {
  g.Vb = g.b[0] * g.b[1] * g.b[2] * g.b[3];
  g.Nb = g.NB[0] * g.NB[1] * g.NB[2] * g.NB[3];
  g.V = (long)g.Vb * g.Nb;
  g.h_loc_nbr.assign(8 * g.Vb, 0);
  g.h_loc_coord.assign(g.Vb, 0);
  for (int loc = 0; loc < g.Vb; loc++) {
    int c[4];
    loc_coords(g.b, loc, c);
    if (loc_index(g.b, c) != loc) throw Error(DDTM_ERR_ARG, "internal: block index map is not a bijection");
    g.h_loc_coord[loc] = c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24);
    for (int k = 0; k < 8; k++) {
      int mu = k / 2, dir = (k & 1) ? -1 : 1;
      int n[4] = {c[0], c[1], c[2], c[3]};
      n[mu] += dir;
      uint32_t cross = 0;
      if (n[mu] < 0 || n[mu] >= g.b[mu]) {
        cross = 1;
        n[mu] = (n[mu] + g.b[mu]) % g.b[mu];
      }
      g.h_loc_nbr[k * g.Vb + loc] = (uint32_t)loc_index(g.b, n) | (cross << 16);
    }
  }
  g.h_blk_nbr.assign(8 * g.Nb, 0);
  for (int blk = 0; blk < g.Nb; blk++) {
    int c[4];
    canon_coords(g.NB, blk, c);
    for (int k = 0; k < 8; k++) {
      int mu = k / 2, dir = (k & 1) ? -1 : 1;
      int n[4] = {c[0], c[1], c[2], c[3]};
      n[mu] += dir;
      int flip = 0;
      if (n[mu] < 0 || n[mu] >= g.NB[mu]) {
        if (mu == 0 && g.bc_t == 1) flip = 1;
        n[mu] = (n[mu] + g.NB[mu]) % g.NB[mu];
      }
      g.h_blk_nbr[k * g.Nb + blk] = canon_index(g.NB, n) | (flip << 30);
    }
  }
  std::vector<int> cb;
  for (int colour = 0; colour < 2; colour++)
    for (int blk = 0; blk < g.Nb; blk++) {
      int c[4];
      canon_coords(g.NB, blk, c);
      if (((c[0] + c[1] + c[2] + c[3]) & 1) == colour) cb.push_back(blk);
    }
  if ((int)cb.size() != g.Nb || g.Nb % 2) throw Error(DDTM_ERR_ARG, "internal: block colouring");
  g.colour_blocks.ensure(cb.size() * 4);
  CK(cudaMemcpy(g.colour_blocks.p, cb.data(), cb.size() * 4, cudaMemcpyHostToDevice));
  g.loc_nbr.ensure(g.h_loc_nbr.size() * 4);
  g.loc_coord.ensure(g.h_loc_coord.size() * 4);
  g.blk_nbr.ensure(g.h_blk_nbr.size() * 4);
  CK(cudaMemcpy(g.loc_nbr.p, g.h_loc_nbr.data(), g.h_loc_nbr.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(g.loc_coord.p, g.h_loc_coord.data(), g.h_loc_coord.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(g.blk_nbr.p, g.h_blk_nbr.data(), g.h_blk_nbr.size() * 4, cudaMemcpyHostToDevice));
}

void build_coarse_geometry(const FineGeom& g, CoarseLevel& c) { build_coarse_geometry_lat(g.NB, c); }

void build_level1_aggregates(const CoarseLevel& c1, const int b[4], Level1Agg& a) {
  a.Vb = 1;
  a.Nagg = 1;
  for (int m = 0; m < 4; m++) {
    if (b[m] < 1 || c1.lat[m] % b[m]) throw Error(DDTM_ERR_ARG, "level-1 block extents must divide the level-1 lattice");
    a.b[m] = b[m];
    a.NB[m] = c1.lat[m] / b[m];
    if (a.NB[m] % 2) throw Error(DDTM_ERR_ARG, "level-1 blocks per direction must be even (red-black SAP)");
    a.Vb *= b[m];
    a.Nagg *= a.NB[m];
  }
  a.h_sites.assign((size_t)a.Nagg * a.Vb, 0);
  std::vector<int> col[2];
  for (int A = 0; A < a.Nagg; A++) {
    int B[4];
    canon_coords(a.NB, A, B);
    col[(B[0] + B[1] + B[2] + B[3]) & 1].push_back(A);
    for (int q = 0; q < a.Vb; q++) {
      int o[4], x[4];
      canon_coords(a.b, q, o);
      for (int m = 0; m < 4; m++) x[m] = B[m] * a.b[m] + o[m];
      a.h_sites[(size_t)A * a.Vb + q] = canon_index(c1.lat, x);
    }
  }
  a.sites.ensure(a.h_sites.size() * 4);
  CK(cudaMemcpy(a.sites.p, a.h_sites.data(), a.h_sites.size() * 4, cudaMemcpyHostToDevice));
  std::vector<int> cl(col[0]);
  cl.insert(cl.end(), col[1].begin(), col[1].end());
  a.colour.ensure(cl.size() * 4);
  CK(cudaMemcpy(a.colour.p, cl.data(), cl.size() * 4, cudaMemcpyHostToDevice));
  // Galerkin parts (level1.cu): table t = 0 keeps the hops that stay inside the aggregate, table
  // t = 1 + k only hop k where it leaves the aggregate; every other hop reads the zero site Nc1
  const int Nc = c1.Nc;
  std::vector<int> agg_of(Nc);
  for (int A = 0; A < a.Nagg; A++)
    for (int q = 0; q < a.Vb; q++) agg_of[a.h_sites[(size_t)A * a.Vb + q]] = A;
  std::vector<int> tabs((size_t)9 * 8 * Nc);
  for (int t = 0; t < 9; t++)
    for (int k = 0; k < 8; k++)
      for (int i = 0; i < Nc; i++) {
        const int nb = c1.h_nbr[(size_t)k * Nc + i];
        const bool cross = agg_of[nb] != agg_of[i];  // NB >= 2 in every direction
        const bool keep = t == 0 ? !cross : (k == t - 1 && cross);
        tabs[((size_t)t * 8 + k) * Nc + i] = keep ? nb : Nc;
      }
  a.tabs.ensure(tabs.size() * 4);
  CK(cudaMemcpy(a.tabs.p, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice));
  a.geom = true;
}

void build_coarse_geometry_lat(const int lat[4], CoarseLevel& c) {
  c.Nc = 1;
  for (int m = 0; m < 4; m++) {
    c.lat[m] = lat[m];
    c.Nc *= lat[m];
  }
  c.h_nbr.assign(8 * c.Nc, 0);
  c.h_even.clear();
  c.h_odd.clear();
  for (int i = 0; i < c.Nc; i++) {
    int x[4];
    canon_coords(c.lat, i, x);
    ((x[0] + x[1] + x[2] + x[3]) & 1 ? c.h_odd : c.h_even).push_back(i);
    for (int k = 0; k < 8; k++) {
      int mu = k / 2, dir = (k & 1) ? -1 : 1;
      int n[4] = {x[0], x[1], x[2], x[3]};
      n[mu] = (n[mu] + dir + c.lat[mu]) % c.lat[mu];
      c.h_nbr[k * c.Nc + i] = canon_index(c.lat, n);
    }
  }
  std::vector<int> pos(c.Nc);
  for (size_t i = 0; i < c.h_even.size(); i++) pos[c.h_even[i]] = (int)i;
  for (size_t i = 0; i < c.h_odd.size(); i++) pos[c.h_odd[i]] = (int)i;
  int ne = (int)c.h_even.size(), no = (int)c.h_odd.size();
  c.h_nbr_oe.assign(8 * (size_t)no, 0);
  c.h_nbr_eo.assign(8 * (size_t)ne, 0);
  for (int k = 0; k < 8; k++) {
    for (int i = 0; i < no; i++) c.h_nbr_oe[(size_t)k * no + i] = pos[c.h_nbr[(size_t)k * c.Nc + c.h_odd[i]]];
    for (int i = 0; i < ne; i++) c.h_nbr_eo[(size_t)k * ne + i] = pos[c.h_nbr[(size_t)k * c.Nc + c.h_even[i]]];
  }
  c.nbr_oe.ensure(c.h_nbr_oe.size() * 4 + 4);
  c.nbr_eo.ensure(c.h_nbr_eo.size() * 4 + 4);
  CK(cudaMemcpy(c.nbr_oe.p, c.h_nbr_oe.data(), c.h_nbr_oe.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.nbr_eo.p, c.h_nbr_eo.data(), c.h_nbr_eo.size() * 4, cudaMemcpyHostToDevice));
  c.nbr.ensure(c.h_nbr.size() * 4);
  c.even.ensure(c.h_even.size() * 4 + 4);
  c.odd.ensure(c.h_odd.size() * 4 + 4);
  CK(cudaMemcpy(c.nbr.p, c.h_nbr.data(), c.h_nbr.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.even.p, c.h_even.data(), c.h_even.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c.odd.p, c.h_odd.data(), c.h_odd.size() * 4, cudaMemcpyHostToDevice));
}

// ---- twisted boundary conditions as boundary-link phases --------------------------
// A hop that wraps forward in direction mu reads exp(i theta_mu) psi, one that wraps backward
// exp(-i theta_mu) psi; both are the hops of the links U_mu(x) at x_mu = L_mu - 1, so multiplying those
// links by exp(i theta_mu) gives the twisted operator (closed loops, hence the clover term, unchanged).
struct PhaseMap {
  int L[4], b[4], NB[4], Vb, Nb;
  double c[4], s[4];
  const uint32_t* loc_coord;
};
__global__ void k_link_phases(double2* __restrict__ U, PhaseMap m) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)m.Vb * m.Nb) return;
  const int blk = (int)(t / m.Vb), loc = (int)(t - (long)blk * m.Vb);
  int B[4], r = blk;
  B[1] = r % m.NB[1]; r /= m.NB[1];
  B[2] = r % m.NB[2]; r /= m.NB[2];
  B[3] = r % m.NB[3];
  B[0] = r / m.NB[3];
  const uint32_t lc = m.loc_coord[loc];
  for (int mu = 0; mu < 4; mu++) {
    const int x = B[mu] * m.b[mu] + (int)((lc >> (8 * mu)) & 255);
    if (x != m.L[mu] - 1 || (m.c[mu] == 1.0 && m.s[mu] == 0.0)) continue;
    double2* u = U + ((size_t)(blk * 4 + mu) * 9) * m.Vb + loc;
    for (int k = 0; k < 9; k++) {
      const double2 a = u[(size_t)k * m.Vb];
      u[(size_t)k * m.Vb] = make_double2(m.c[mu] * a.x - m.s[mu] * a.y, m.c[mu] * a.y + m.s[mu] * a.x);
    }
  }
}

void launch_link_phases(const FineGeom& g, double* links, const double phase[4], cudaStream_t s) {
  PhaseMap m;
  for (int i = 0; i < 4; i++) {
    m.L[i] = g.L[i];
    m.b[i] = g.b[i];
    m.NB[i] = g.NB[i];
    m.c[i] = cos(phase[i]);
    m.s[i] = sin(phase[i]);
  }
  m.Vb = g.Vb;
  m.Nb = g.Nb;
  m.loc_coord = g.loc_coord.as<uint32_t>();
  k_link_phases<<<(unsigned)((g.V + 127) / 128), 128, 0, s>>>((double2*)links, m);
  CKL("link_phases");
}

// ---- canonical <-> internal ------------------------------------------------------
struct CanonMap {
  int L[4], b[4], NB[4];
  int Vb, Nb;
  const uint32_t* loc_coord;
};

static CanonMap make_map(const FineGeom& g) {
  CanonMap m;
  for (int i = 0; i < 4; i++) { m.L[i] = g.L[i]; m.b[i] = g.b[i]; m.NB[i] = g.NB[i]; }
  m.Vb = g.Vb;
  m.Nb = g.Nb;
  m.loc_coord = g.loc_coord.as<uint32_t>();
  return m;
}

__device__ __forceinline__ size_t canon_site(const CanonMap& m, int blk, int loc) {
  int B[4];
  int r = blk;
  B[1] = r % m.NB[1]; r /= m.NB[1];
  B[2] = r % m.NB[2]; r /= m.NB[2];
  B[3] = r % m.NB[3];
  B[0] = r / m.NB[3];
  uint32_t lc = __ldg(m.loc_coord + loc);
  int t = B[0] * m.b[0] + (lc & 255);
  int x = B[1] * m.b[1] + ((lc >> 8) & 255);
  int y = B[2] * m.b[2] + ((lc >> 16) & 255);
  int z = B[3] * m.b[3] + ((lc >> 24) & 255);
  return (((size_t)t * m.L[3] + z) * m.L[2] + y) * m.L[1] + x;
}

template <int P>
__global__ void k_spinor_from_canon(Spinor<P> out, const double2* __restrict__ in, CanonMap m) {
  typedef typename Prec<P>::real R;
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)m.Vb * m.Nb) return;
  int blk = (int)(s / m.Vb), loc = (int)(s - (long)blk * m.Vb);
  size_t i = canon_site(m, blk, loc);
  cplx<R> v[12];
#pragma unroll
  for (int c = 0; c < 12; c++) {
    double2 a = in[i * 12 + c];
    v[c] = cplx<R>((R)a.x, (R)a.y);
  }
  out.store(blk, loc, v);
}

template <int P>
__global__ void k_spinor_to_canon(Spinor<P> in, double2* __restrict__ out, CanonMap m) {
  typedef typename Prec<P>::real R;
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)m.Vb * m.Nb) return;
  int blk = (int)(s / m.Vb), loc = (int)(s - (long)blk * m.Vb);
  size_t i = canon_site(m, blk, loc);
  cplx<R> v[12];
  in.loadw(blk, loc, v);
#pragma unroll
  for (int c = 0; c < 12; c++) out[i * 12 + c] = make_double2((double)v[c].re, (double)v[c].im);
}

__global__ void k_links_from_canon(double2* __restrict__ out, const double2* __restrict__ U, CanonMap m) {
  long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= (long)m.Vb * m.Nb) return;
  int blk = (int)(s / m.Vb), loc = (int)(s - (long)blk * m.Vb);
  size_t i = canon_site(m, blk, loc);
  for (int mu = 0; mu < 4; mu++)
    for (int k = 0; k < 9; k++) out[(((size_t)blk * 4 + mu) * 9 + k) * m.Vb + loc] = U[(i * 4 + mu) * 9 + k];
}

static unsigned grid_for(long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

void launch_spinor_from_canon(const FineGeom& g, int prec, void* d, float* nrm, const double* in, cudaStream_t s) {
  ScopedTimer timer_("layout_in", s);
  CanonMap m = make_map(g);
  unsigned grid = grid_for(g.V, 128);
  const double2* src = reinterpret_cast<const double2*>(in);
  if (prec == PREC_F64) {
    Spinor<PREC_F64> o{(double2*)d, nullptr, g.Vb};
    k_spinor_from_canon<PREC_F64><<<grid, 128, 0, s>>>(o, src, m);
  } else if (prec == PREC_F32) {
    Spinor<PREC_F32> o{(float2*)d, nullptr, g.Vb};
    k_spinor_from_canon<PREC_F32><<<grid, 128, 0, s>>>(o, src, m);
  } else {
    Spinor<PREC_F16> o{(__half2*)d, nrm, g.Vb};
    k_spinor_from_canon<PREC_F16><<<grid, 128, 0, s>>>(o, src, m);
  }
  CKL("spinor_from_canon");
}

void launch_spinor_to_canon(const FineGeom& g, int prec, const void* d, const float* nrm, double* out, cudaStream_t s) {
  ScopedTimer timer_("layout_out", s);
  CanonMap m = make_map(g);
  unsigned grid = grid_for(g.V, 128);
  double2* dst = reinterpret_cast<double2*>(out);
  if (prec == PREC_F64) {
    Spinor<PREC_F64> i{(double2*)d, nullptr, g.Vb};
    k_spinor_to_canon<PREC_F64><<<grid, 128, 0, s>>>(i, dst, m);
  } else if (prec == PREC_F32) {
    Spinor<PREC_F32> i{(float2*)d, nullptr, g.Vb};
    k_spinor_to_canon<PREC_F32><<<grid, 128, 0, s>>>(i, dst, m);
  } else {
    Spinor<PREC_F16> i{(__half2*)d, (float*)nrm, g.Vb};
    k_spinor_to_canon<PREC_F16><<<grid, 128, 0, s>>>(i, dst, m);
  }
  CKL("spinor_to_canon");
}

void launch_links_from_canon(const FineGeom& g, double* out, const double* U, cudaStream_t s) {
  CanonMap m = make_map(g);
  k_links_from_canon<<<grid_for(g.V, 128), 128, 0, s>>>((double2*)out, (const double2*)U, m);
  CKL("links_from_canon");
}

__global__ void k_convert_f32(const double2* __restrict__ in, float2* __restrict__ out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { double2 a = in[i]; out[i] = make_float2((float)a.x, (float)a.y); }
}
__global__ void k_convert_f16(const double2* __restrict__ in, __half2* __restrict__ out, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { double2 a = in[i]; out[i] = __floats2half2_rn((float)a.x, (float)a.y); }
}

void launch_convert_complex(const double* in, int prec_out, void* out, size_t n, cudaStream_t s) {
  unsigned grid = grid_for((long)n, 256);
  if (prec_out == PREC_F32) k_convert_f32<<<grid, 256, 0, s>>>((const double2*)in, (float2*)out, n);
  else if (prec_out == PREC_F16) k_convert_f16<<<grid, 256, 0, s>>>((const double2*)in, (__half2*)out, n);
  else CK(cudaMemcpyAsync(out, in, n * 16, cudaMemcpyDeviceToDevice, s));
  CKL("convert_complex");
}

__global__ void k_count_nonfinite(const double* __restrict__ a, size_t n, int* counter) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  int bad = (i < n) && !isfinite(a[i]);
  bad = __syncthreads_count(bad);
  if (threadIdx.x == 0 && bad) atomicAdd(counter, bad);
}

void launch_count_nonfinite(const double* a, size_t n, int* counter, cudaStream_t s) {
  k_count_nonfinite<<<grid_for((long)n, 256), 256, 0, s>>>(a, n, counter);
  CKL("count_nonfinite");
}

}  // namespace ddtm

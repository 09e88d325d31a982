// Launch shape of the SIMT coarse stencil kernels (k_coarse_apply,
// k_coarse_even in coarse.cu).  Plain host C++, no CUDA types, so that a host
// unit test can compile it alone and check every (n, R) it may meet.
//
// A site of the coarse lattice (n = 2 nv rows) with R right-hand sides is
// worked on by n/2 row pairs x G chunk slots; a thread owns one row pair and
// the RHS chunks ch = g, g + G, g + 2G, ... of RC consecutive right-hand sides
// each.  CTAs hold whole sites and at most kMaxThreads threads.
#pragma once

namespace ddtm {

struct CoarseShape {
  int rc;       // right-hand sides per chunk (4, 2 or 1: the largest that divides R)
  int nch;      // chunks per site, R / rc
  int groups;   // chunk slots per row pair (G); a thread loops over nch / G chunks
  int per;      // threads per site, n/2 * G
  int spb;      // sites per CTA
  int threads;  // threads per CTA, spb * per
};

static const int kCoarseMaxThreads = 256;  // the kernels' __launch_bounds__

inline CoarseShape coarse_shape(int n, int R) {
  CoarseShape s;
  s.rc = (R % 4 == 0) ? 4 : (R % 2 == 0) ? 2 : 1;
  s.nch = R / s.rc;
  const int np = n / 2;
  int gmax = kCoarseMaxThreads / np;
  if (gmax < 1) gmax = 1;
  s.groups = s.nch < gmax ? s.nch : gmax;
  s.per = np * s.groups;
  s.spb = s.per >= kCoarseMaxThreads ? 1 : kCoarseMaxThreads / s.per;
  s.threads = s.spb * s.per;
  return s;
}

}  // namespace ddtm

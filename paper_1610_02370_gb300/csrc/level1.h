// Host interface of the intermediate-level kernels of a three-level hierarchy (level1.cu).
#pragma once

#include "common.cuh"
#include "ddtm_internal.h"

namespace ddtm {

// P_1 from the level-1 test vectors a.tv (classical Gram-Schmidt twice per aggregate half)
void launch_l1_build_P(Level1Agg& a, const CoarseLevel& c1, cudaStream_t st);
// c = P_1^+ v (level 1 -> level 2) and v (+)= P_1 c (level 2 -> level 1) on interleaved batches of
// stride R, for the first Rv right-hand sides
void launch_l1_restrict(const Level1Agg& a, const CoarseLevel& c1, float2* c, const float2* v, int R, int Rv,
                        cudaStream_t st);
void launch_l1_prolong(const Level1Agg& a, const CoarseLevel& c1, float2* v, const float2* c, int R, int Rv, int add,
                       cudaStream_t st);
// D_2 = P_1^+ D_1 P_1 into c2.Dc (the twist is added on the fly, as on every coarse level)
void launch_l1_galerkin(const Level1Agg& a, const CoarseLevel& c1, CoarseLevel& c2, ScratchPool& pool, cudaStream_t st);
// one half-sweep of the red-black SAP smoother on D_1(mu) over the aggregates of one colour (0 red,
// 1 black), x updated in place; R a multiple of 4
void launch_l1_sap_half(const Level1Agg& a, const CoarseLevel& c1, float2* x, const float2* b, int colour, double mu,
                        int nmr, int R, cudaStream_t st);

// nsep separate vectors of N complex entries (sep[r * N + e]) <-> an interleaved batch of R >= nsep
// (inter[e * R + r]); dir 0 fills the padding columns with zeros
void launch_l1_transpose(float2* sep, float2* inter, size_t N, int nsep, int R, int dir, cudaStream_t st);

}  // namespace ddtm

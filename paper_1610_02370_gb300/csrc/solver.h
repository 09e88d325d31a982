// Host-side multigrid and solver internals shared between the C ABI and the
// solver implementation.
#pragma once

#include "ddtm_internal.h"

namespace ddtm {

// largest batch of right-hand sides one outer solve carries in lockstep (the
// interleaved coarse vectors of a batch hold at most this many columns)
static const int kMaxBatch = 256;

size_t store2_bytes(int prec);
void check_prec(int prec);
void check_loc(int loc);
void require_gauge(ddtm_ctx* c);
void ensure_fine_prec(ddtm_ctx* c, int prec);
void ensure_site_inverse(ddtm_ctx* c, int prec, double mu);
const double* stage_in(ddtm_ctx* c, const char* name, const double* x, size_t ncomplex, int loc);
double* stage_out(ddtm_ctx* c, const char* name, double* y, size_t ncomplex, int loc);
void unstage_out(ddtm_ctx* c, double* y, const double* d, size_t ncomplex, int loc);
void field_alloc(ddtm_field* f);
void* field_ptr(const ddtm_field* f, int r);
float* field_nrm(const ddtm_field* f, int r);
void dslash_field(ddtm_ctx* c, ddtm_field* y, const ddtm_field* x, double mu);

// ncycles red-black SAP cycles on D(mu) x = b (from x = 0 if from_zero) for R
// right-hand sides: fields of precision prec at stride 12 V, FP16 scales at stride V.
void sap_run(ddtm_ctx* c, int prec, void* x, float* xn, const void* b, const float* bn, double mu, int ncycles,
             int nmr, bool from_zero, int R);

void validate_params(ddtm_ctx* c, const ddtm_params& p);
void invalidate_setup(ddtm_ctx* c);

}  // namespace ddtm

/*
 * ddtm.h -- C ABI of libddtm, the GB300 hot path of twisted-mass DD-alpha-AMG
 * (Alexandrou, Bacchio, Finkenrath, Frommer, Kahl, Rottmann, arXiv:1610.02370).
 *
 * The library solves D(mu) psi = b with D(mu) = D_W + i mu Gamma5, the clover
 * Wilson-Dirac operator with a twisted mass (Sec. 2.1), by flexible GMRES
 * preconditioned with the aggregation-based multigrid of Sec. 2.2-2.6.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Normalisation (Sec. 2.1): D_W = (m+4) I - c_sw/32 sum (gamma gamma) x (Q - Q)
 *   - 1/2 sum [(1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)],
 *   m = 1/(2 kappa) - 4, twist i mu Gamma5 with mu used as given.
 * Gamma basis: chiral, gamma_0 = [[0,1],[1,0]], gamma_k = [[0, i s_k], [-i s_k, 0]]
 *   (k = 1, 2, 3 for x, y, z), so gamma5 = gamma_0 gamma_1 gamma_2 gamma_3 =
 *   diag(1, 1, -1, -1) as printed in Sec. 2.1.
 * Directions: mu = 0 (t), 1 (x), 2 (y), 3 (z).  dims[] = {T, X, Y, Z}.
 * Canonical layout of every host/device array passed in or out: complex
 *   FP64 interleaved (re, im); site index ((t*Lz + z)*Ly + y)*Lx + x;
 *   gauge field U[site][mu][row][col]; spinor [rhs][site][spin][colour];
 *   coarse vector [rhs][coarse site][s*Nv + i], coarse sites in the same
 *   canonical order over the block lattice, s = 0 for the Gamma5 = +1
 *   aggregate half (spins 0, 1), s = 1 for spins 2, 3 (Sec. 2.3).
 * Location: loc = DDTM_LOC_HOST (pointers are host memory, copied in/out)
 *   or DDTM_LOC_DEVICE (pointers are device memory of the context's GPU, e.g.
 *   torch.Tensor.data_ptr()).  The caller owns its buffers; the library owns
 *   all of its internal device state.
 * Precision prec: DDTM_PREC_F64 (FP64 storage and arithmetic), DDTM_PREC_F32,
 *   DDTM_PREC_F16 (FP16 storage with one FP32 scale per site for spinors,
 *   FP32 arithmetic).
 * Errors: every function returns DDTM_OK (0) or a negative DDTM_ERR_* code;
 *   ddtm_last_error() gives the message of the last failure on a context.
 *   Calls out of order (e.g. solve before setup) return DDTM_ERR_STATE.
 * Streams: all work is issued on the context's stream (ddtm_set_stream);
 *   calls that return host-visible results synchronise that stream.
 * Threads: a context must not be used by two threads at once.
 */
#ifndef DDTM_H
#define DDTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDTM_OK 0
#define DDTM_ERR_ARG (-1)     /* invalid argument (sizes, pointers, enum values) */
#define DDTM_ERR_CUDA (-2)    /* CUDA runtime error */
#define DDTM_ERR_OOM (-3)     /* device allocation failed */
#define DDTM_ERR_NOCONV (-4)  /* solver stopped before reaching its tolerance */
#define DDTM_ERR_NAN (-5)     /* NaN/Inf met in a norm or input */
#define DDTM_ERR_STATE (-6)   /* call order: gauge, setup or coarse operator missing */
#define DDTM_ERR_TIMEOUT (-7) /* a bounded device-side wait gave up */

#define DDTM_LOC_HOST 0
#define DDTM_LOC_DEVICE 1

#define DDTM_PREC_F64 0
#define DDTM_PREC_F32 1
#define DDTM_PREC_F16 2

#define DDTM_MAX_LEVELS 4

typedef struct ddtm_ctx ddtm_ctx;
typedef struct ddtm_field ddtm_field;

/* Multigrid and solver parameters; defaults (ddtm_default_params) are the
 * parameter set of Table 1, except n_levels = 2.  Level l = 0 is the fine
 * lattice; block[l] is the aggregate (= SAP block, Sec. 2.4) of level l and
 * nv[l] the number of test vectors that build level l+1. */
typedef struct {
  int n_levels;            /* 2 or 3 */
  int n_setup;             /* setup iterations (Sec. 2.6), Table 1: 5 */
  int nv[DDTM_MAX_LEVELS]; /* test vectors per level, Table 1: 28, 28 */
  int block[DDTM_MAX_LEVELS][4]; /* block extents {t, x, y, z}, Table 1: 4^4 then 2^4 */
  int post_smooth;         /* SAP cycles after the coarse correction, Table 1: 4 */
  int nmr;                 /* MR steps per block solve, Table 1: 3 */
  int kcycle_restart;      /* K-cycle FGMRES (levels 1..L-2), Table 1: 5 */
  int kcycle_max_restarts; /* Table 1: 2 */
  double kcycle_tol;       /* Table 1: 1e-1 */
  int coarse_restart;      /* coarsest even-odd GMRES, Table 1: 100 */
  int coarse_max_restarts; /* Table 1: 5 */
  double coarse_tol;       /* Table 1: 1e-1 */
  double delta;            /* coarsest twist mu_c = delta * mu (Sec. 2.3), Table 1: 5.2 */
  int outer_restart;       /* outer FGMRES restart length, 30 */
  int outer_max_iters;     /* cap on outer iterations over all restarts */
  double outer_tol;        /* relative residual ||b - D x|| / ||b||, 1e-10 */
  double restart_tol;      /* mixed-precision restart criterion, Table 1: 1e-6 */
  int smoother_prec;       /* storage precision of SAP and transfer: DDTM_PREC_F16 or F32 (mixed-precision
                              outer cycle in FP32), or DDTM_PREC_F64 (the whole fine level in FP64: the plain
                              FP64 method; the coarse correction stays FP32) */
  int coarse_prec;         /* coarse operator: DDTM_PREC_F32 (FP32 blocks, SIMT stencil) or DDTM_PREC_F16
                              (FP16 operand images on the tensor cores, FP32 accumulation, FP16 Krylov
                              basis in the coarsest GMRES) */
} ddtm_params;

/* Per-solve report (Tables 2-3 columns): iteration counts, residuals, times. */
typedef struct {
  int iters;          /* outer FGMRES iterations (max over right-hand sides) */
  int restarts;       /* outer restarts with an FP64 residual recomputation */
  long coarse_iters;  /* total coarsest-level GMRES iterations */
  double max_relres;  /* max over rhs of ||b - D x|| / ||b|| (FP64 operator) */
  double solve_s;     /* wall time of the solve */
  double setup_s;     /* wall time of the last setup */
} ddtm_solve_info;

/* ---- context ------------------------------------------------------------ */

/* Create a context on the current CUDA device for a T x X x Y x Z lattice.
 * dims = {T, X, Y, Z}; block = {bt, bx, by, bz} fine aggregate / SAP block
 * (NULL: 4^4).  Every block extent must be even and divide its lattice
 * extent, and the number of blocks per direction must be even (red-black
 * block colouring, Sec. 2.4).  bc_t: 0 periodic, 1 antiperiodic in t for
 * the fermion hops (the paper leaves boundary conditions to the library).
 * Returns DDTM_ERR_ARG on invalid sizes; *out is NULL on failure. */
int ddtm_create(ddtm_ctx** out, const int dims[4], const int block[4], int bc_t);
int ddtm_destroy(ddtm_ctx* ctx);
/* Message of the last failing call on ctx ("" if none); owned by ctx. */
const char* ddtm_last_error(ddtm_ctx* ctx);
/* Issue all further work on this cudaStream_t (NULL: the legacy default stream). */
int ddtm_set_stream(ddtm_ctx* ctx, void* cuda_stream);
/* Fill p with the defaults described at ddtm_params. */
int ddtm_default_params(ddtm_params* p);
/* Copy the context's current parameters (defaults with block[0] set to the
 * block of ddtm_create until ddtm_set_params is called) into *p. */
int ddtm_get_params(ddtm_ctx* ctx, ddtm_params* p);
/* Validate and store parameters.  Changing block[0] after ddtm_create is
 * rejected (DDTM_ERR_ARG): it fixes the internal layout. */
int ddtm_set_params(ddtm_ctx* ctx, const ddtm_params* p);

/* ---- fine operator (Sec. 2.1) -------------------------------------------- */

/* Load the gauge field U (canonical layout, V*4*9 complex) and build the
 * clover site term from the four-leaf Q_mu_nu of Sec. 2.1 with
 * m = 1/(2 kappa) - 4.  Invalidates any setup.  DDTM_ERR_NAN if U holds a
 * NaN/Inf. */
int ddtm_load_gauge(ddtm_ctx* ctx, const double* U, int loc, double kappa, double c_sw);

/* Twisted boundary conditions psi(x + L_mu mu_hat) = exp(i theta_mu) psi(x)
 * for mu = t, x, y, z (a library feature the paper lists for its HMC use,
 * Sec. 3.2 and the appendix): applied to the links U_mu(x) at x_mu = L_mu - 1
 * (the clover term, built from closed loops, is unchanged), on top of the
 * antiperiodic t of ddtm_create.  May be called before or after
 * ddtm_load_gauge; a change invalidates the setup.  theta = {0, 0, 0, 0}
 * restores periodic boundaries. */
int ddtm_set_boundary_phases(ddtm_ctx* ctx, const double theta[4]);

/* y = D(mu) x for nrhs right-hand sides (canonical spinors), computed in
 * storage precision prec (Sec. 2.1; mu may be +mu or -mu, the two flavours). */
int ddtm_apply_D(ddtm_ctx* ctx, double* y, const double* x, int nrhs, double mu, int prec, int loc);

/* x = ncycles red-black SAP cycles on D(mu) x = b from x = 0 (Sec. 2.4):
 * each cycle updates the red blocks, then the black blocks, each with nmr
 * minimal-residual steps on the even-odd reduced block system and Dirichlet
 * block boundaries.  Block size = block[0]. */
int ddtm_sap(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu, int ncycles, int nmr,
             int prec, int loc);

/* y = D(mu) x like ddtm_apply_D, for one right-hand side held in device
 * memory (canonical layout), without allocating anything during the call.
 * Meant for callers that cannot call cudaMalloc: cudaMalloc and cudaFree may
 * synchronise the whole device and stall their other streams, or the caller's
 * own allocator already owns the device memory budget.  The paper has no
 * counterpart; it is an interface convenience around the Sec. 2.1 operator.
 * Working memory: one fixed 64 MiB device array inside the library (held by
 * every GPU that loads the library until the process exits), enough for two
 * internal-layout fields of up to 174762 sites in FP64 (e.g. 16^3 x 32);
 * larger lattices return DDTM_ERR_ARG with the sizes in the message.  The
 * first call on a device looks up the array's device address; make that call
 * before any stream capture.  All calls share the array, which keeps the last
 * call's contents (every byte a call reads it writes first), so calls that
 * overlap on the GPU race.  Work is issued on the context's stream and not
 * synchronised.  x and y must be distinct device pointers; the gauge field
 * must already be held in precision prec (FP64 always is; one ddtm_apply_D
 * call with F32 or F16 creates that copy), else DDTM_ERR_STATE. */
int ddtm_apply_D_noalloc(ddtm_ctx* ctx, double* y, const double* x, double mu, int prec);

/* ---- device-resident fine fields (internal layout) ------------------------ */

/* A fine spinor field of nrhs right-hand sides held on the device in the
 * library's internal even-odd block layout and precision prec.  Lets callers
 * chain operator applications without host round trips. */
int ddtm_field_create(ddtm_ctx* ctx, int prec, int nrhs, ddtm_field** out);
int ddtm_field_destroy(ddtm_field* f);
/* Convert canonical FP64 spinors (nrhs of them) into / out of a field. */
int ddtm_field_import(ddtm_ctx* ctx, ddtm_field* f, const double* x, int loc);
int ddtm_field_export(ddtm_ctx* ctx, const ddtm_field* f, double* x, int loc);
/* y = D(mu) x on fields of equal precision and nrhs (Sec. 2.1). */
int ddtm_apply_D_field(ddtm_ctx* ctx, ddtm_field* y, const ddtm_field* x, double mu);
/* x = SAP(b) as in ddtm_sap, on fields of equal precision (F64, F32 or F16) and nrhs; all
 * right-hand sides go through one launch per half-sweep. */
int ddtm_sap_field(ddtm_ctx* ctx, ddtm_field* x, const ddtm_field* b, double mu, int ncycles, int nmr);

/* ---- aggregation and coarse levels (Sec. 2.3) ------------------------------ */

/* Adaptive setup (Sec. 2.6): random test vectors (counter-based generator
 * keyed by seed), one SAP pass, then n_setup - 1 inverse-iteration steps with
 * the current multigrid; P and the coarse operators are rebuilt after each. */
int ddtm_setup(ddtm_ctx* ctx, double mu, uint64_t seed);

/* Update an existing setup (the HMC usage of Sec. 3.2: after the gauge field
 * (ddtm_load_gauge) or the twist changed): the test vectors of the last
 * setup are kept, P and the coarse operators are rebuilt from them with the
 * current gauge field, and n_iter inverse-iteration steps (Sec. 2.6, k >= 2)
 * at twist mu follow (n_iter = 0: rebuild only).  DDTM_ERR_STATE if no
 * test vectors of the current parameters exist. */
int ddtm_setup_update(ddtm_ctx* ctx, double mu, int n_iter);

/* Replace the test vectors of level `level` (0, or 1 of three levels) by v
 * (nv canonical fine spinors for level 0, nv canonical level-1 coarse vectors
 * for level 1), orthonormalise them per aggregate half (Gamma5-compatible
 * aggregation, Sec. 2.3) into P_level, and build the operator of the next
 * level, D_{level+1} = P^+ D_level P.  Test hook for parity against an
 * independent implementation; nv must equal params.nv[level]; level 1 needs
 * the level-0 vectors first. */
int ddtm_set_test_vectors(ddtm_ctx* ctx, int level, const double* v, int nv, int loc);

/* Rebuild every coarse operator from the current P (Galerkin, Sec. 2.3). */
int ddtm_build_coarse(ddtm_ctx* ctx);

/* P of level 0 in canonical form: array [2][nv] of fine spinors; entry
 * (s, i) restricted to aggregate j is column (j, s, i) of P. */
int ddtm_get_prolongator(ddtm_ctx* ctx, int level, double* W, int loc);

/* c = R x = P^+ x and x = P c between level 0 and level 1 (Sec. 2.3). */
int ddtm_restrict(ddtm_ctx* ctx, int level, double* c, const double* x, int nrhs, int loc);
int ddtm_prolong(ddtm_ctx* ctx, int level, double* x, const double* c, int nrhs, int loc);

/* y = D_level(mu) x on coarse vectors, D_c(mu) = P^+ D P + i mu Gamma5_c
 * (Sec. 2.3); level >= 1.  mu is used as given (pass delta*mu for the
 * shifted coarsest operator).  All nrhs vectors go through one batched
 * stencil pass: FP32 blocks on the SIMT cores (coarse_prec F32), or FP16
 * operand images on the tensor cores with FP32 accumulation (coarse_prec
 * F16; DDTM_ERR_TIMEOUT if a pipeline wait of that kernel gave up). */
int ddtm_apply_Dc(ddtm_ctx* ctx, int level, double* y, const double* x, int nrhs, double mu, int loc);

/* x = ncycles red-black SAP cycles on D_level(mu) x = b from x = 0 on a
 * coarse level (Sec. 2.4 applied to the Galerkin operator, the smoother of
 * the intermediate level of three, Sec. 2.2): the blocks are the level's
 * aggregates (block[level]), each block system (hops leaving the block
 * dropped) gets nmr minimal-residual steps on the full block from zero, red
 * blocks first.  Vectors in the canonical coarse layout of that level.  Test
 * hook; level must be 1 with n_levels = 3 (DDTM_ERR_ARG otherwise). */
int ddtm_sap_coarse(ddtm_ctx* ctx, int level, double* x, const double* b, int nrhs, double mu, int ncycles, int nmr,
                    int loc);

/* Even-odd preconditioned GMRES on the coarsest level (Sec. 2.5) for
 * D_c(mu_c) x = b with mu_c as given; restart length, restarts and tolerance
 * from the parameters (with coarse_prec F16 the Schur complement runs on the
 * tensor cores and the Krylov basis is stored in FP16).  *iters receives the
 * iteration count.  Returns DDTM_ERR_NOCONV if the tolerance was not reached. */
int ddtm_coarse_solve(ddtm_ctx* ctx, double* x, const double* b, double mu_c, int loc, int* iters);

/* The same solve for nrhs right-hand sides at once (arrays of nrhs canonical
 * coarse vectors, contiguous): one batched GMRES whose Krylov kernels and
 * coarse-stencil passes take all of them together, as inside the multigrid
 * solver (the batch is padded with zero columns to the sizes those kernels
 * take).  *iters receives the iteration count of the batch.  Returns
 * DDTM_ERR_NOCONV if any right-hand side missed the tolerance. */
int ddtm_coarse_solve_batch(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu_c, int loc, int* iters);

/* ---- solve (Sec. 2.2, 2.5) ---------------------------------------------------- */

/* Solve D(mu) x = b for nrhs right-hand sides to params.outer_tol (relative,
 * FP64 residual) with flexible GMRES preconditioned by the K-cycle multigrid;
 * mu may be +mu or -mu with one setup (Sec. 3.1).  The right-hand sides are
 * solved in lockstep as one batch (every stencil, smoother and coarse-solve
 * launch covers all of them) unless their outer-solver fields do not fit in
 * the device memory (or exceed 256), in which case they go in batches of the largest size that fits
 * (at most 256).  info
 * may be NULL.  DDTM_ERR_NOCONV (info still filled) if outer_max_iters is
 * exhausted; DDTM_ERR_TIMEOUT if a tensor-core pipeline wait gave up. */
int ddtm_solve(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu, int loc,
               ddtm_solve_info* info);

/* The baseline solver the paper compares with (Sec. 3.1.2): conjugate
 * gradient on the normal equations D_hat^+ D_hat x_o = D_hat^+ rhat of the
 * even-odd Schur complement D_hat = D_oo - D_oe D_ee^-1 D_eo (odd sites; the
 * even sites follow by D_ee^-1), in FP64 on the GPU, one right-hand side
 * after another; needs only the gauge field (no setup).  D_hat^+ is applied
 * as Gamma5 D_hat(-mu) Gamma5.  Each solve stops when the true FP64 relative
 * residual ||b - D(mu) x|| / ||b|| is <= tol (checked after the residual of the
 * normal equations has dropped by tol, and again while it is not) or after
 * max_iter CG iterations (DDTM_ERR_NOCONV, info still filled).  info: iters =
 * CG iterations (max over right-hand sides), max_relres, solve_s. */
int ddtm_eo_cg(ddtm_ctx* ctx, double* x, const double* b, int nrhs, double mu, double tol, int max_iter, int loc,
               ddtm_solve_info* info);

/* Save / load the setup (parameters, mu, test vectors of every level) to a
 * file; loading rebuilds P and the coarse operators. */
int ddtm_save_setup(ddtm_ctx* ctx, const char* path);
int ddtm_load_setup(ddtm_ctx* ctx, const char* path);

/* ---- execution options ---------------------------------------------------------- */

/* Set / read an execution option of the context (results depend on none but
 * the test hook "tc_forced_timeout_us"):
 *   "graphs" (default 1): each iteration of the coarsest even-odd GMRES
 *     (Sec. 2.5; operator passes, Gram-Schmidt, Givens update, residual
 *     estimate) is captured once per iteration index, batch and buffer set
 *     into a CUDA graph and replayed with one launch; 0 launches its kernels
 *     one by one.  Graphs are not used while the per-kernel timers are on.
 *   "graphs_cached" (read only): executable graphs held by the context.
 *   "autotune" (default 1, process-wide): the first launch of each shape of
 *     the tensor-core coarse stencil pass (column groups, rows, outputs)
 *     outside stream capture times every residency its registers allow (1, 2
 *     or 3 CTAs per SM, the stage ring filling the shared memory left per CTA)
 *     and keeps the fastest for that shape; each output is formed by the same
 *     MMAs in the same order in every variant, so results do not change.
 *     0 uses the fixed rule (2 CTAs per SM up to 16 right-hand sides, else 1).
 *   "tc_forced_timeout_us" (default 0, process-wide; a test hook of the
 *     failure path): when v > 0, the MMA thread of every tensor-core pass
 *     first waits v microseconds on a barrier that nothing completes; the
 *     wait runs out, the pass stops (its bulk copies awaited, tensor memory
 *     freed) and the call reports DDTM_ERR_TIMEOUT with its outputs
 *     undefined.  Passes so launched are neither autotuned nor captured into
 *     graphs.  Valid range 0 ... 1000000; set 0 to resume normal operation.
 * DDTM_ERR_ARG for an unknown name or a value out of range. */
int ddtm_set_option(ddtm_ctx* ctx, const char* name, int value);
int ddtm_get_option(ddtm_ctx* ctx, const char* name, int* value);
/* The autotuner's choices so far as a JSON object (NUL-terminated, truncated
 * to len): {"<pass>|n<rows>|R<rhs>|out<outputs>|s<self>|h<hops>":
 * {"ctas_per_sm": k, "ms": [time with 1, 2, ... CTAs per SM]}, ...}. */
int ddtm_autotune_report(char* buf, int len);

/* ---- device memory budget ---------------------------------------------------- */

/* Cap on the device memory the library holds, over all contexts of the
 * process (bytes; 0 removes the cap, the default).  An allocation that would
 * exceed it fails with DDTM_ERR_OOM before cudaMalloc is called, exactly as a
 * failed cudaMalloc does; the call that needed it returns DDTM_ERR_OOM and the
 * context stays usable (a later call may succeed under a larger cap).  Lets a
 * caller that shares the GPU keep the solver within a share of HBM (the paper
 * has no counterpart; it runs one solver per node). */
int ddtm_set_memory_limit(size_t bytes);

/* Frees the context's solver workspace (Krylov bases, batched fields, staging
 * buffers; the cached graphs that refer to them are destroyed) after
 * synchronising its stream.  The gauge field, the hierarchy and the setup
 * stay; the next call that needs workspace allocates it again. */
int ddtm_release_workspace(ddtm_ctx* ctx);
/* Device bytes the library holds now (all contexts and fields). */
int ddtm_memory_in_use(size_t* bytes);

/* ---- measurement ------------------------------------------------------------ */

/* Per-kernel CUDA-event timing (the paper reports its cost in setup and
 * solve time, Tables 2-4; these timers break the GPU time down by kernel).
 * When enabled, every kernel launch of the library is bracketed by two events
 * on its stream.  Timers are process-wide (shared by all contexts). */
int ddtm_timer_enable(ddtm_ctx* ctx, int on);
int ddtm_timer_reset(ddtm_ctx* ctx);
/* Write a JSON object {"_kernel_launches": k, "name": {"launches": n, "ms": total, "units": u,
 * "bytes": b}, ...} into buf (NUL-terminated, truncated to len); synchronises the recorded events.
 * k counts every kernel the library launched since the last reset (timed or not); per name, n
 * counts timed launch scopes, u their work units (right-hand sides or vectors) and b their
 * algorithmic bytes where the library states them (0 otherwise). */
int ddtm_timer_report(ddtm_ctx* ctx, char* buf, int len);

/* Measured arithmetic peak of the current device's SIMT units: fused
 * multiply-add throughput (2 flops each) in FP64 (prec = DDTM_PREC_F64) or
 * FP32 (DDTM_PREC_F32), from a kernel of independent FMA chains on every SM,
 * timed with CUDA events (best of four launches after two warm-ups) at the
 * clocks the GPU runs at.  The roofline of the ALU-bound kernels is taken
 * against it (the paper reports no device peaks).  *ms receives the best
 * launch time and *sm_count the device's SM count (either may be NULL).
 * DDTM_ERR_ARG for another prec; synchronises the device. */
int ddtm_measure_fma_peak(int prec, double* flops_per_s, double* ms, int* sm_count);

#ifdef __cplusplus
}
#endif

#endif /* DDTM_H */

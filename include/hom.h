/*
 * hom.h — C ABI of the GB300 Fourier-Galerkin homogenization library (libhom).
 *
 * The library solves the discrete corrector problems of Mishra, Vondrejc & Zeman,
 * "A comparative study on low-memory iterative solvers for FFT-based homogenization of
 * periodic media" (arXiv:1508.02045), on one CUDA GPU:
 *
 *   (A_H E, E) = min over e in E_N of a(E + e, E + e)                 Section 2, eq. (homog_form)
 *   C x = b,  C = G A,  b = -G A E                                     Section 2.3, eq. (linsys)
 *
 * with G = F^{-1} Gamma^ F the projection of eq. (discrete_proj), Gamma^(k) = k k^T / (k.k),
 * Gamma^(0) = 0 (eq. (proj)), and A either sampled at the grid nodes (GaNi, Section 2.2) or
 * assembled on the double grid M = 2N - 1 from its Fourier coefficients (Ga, eq.
 * (Ga_exact_integration)). The four solvers are Algorithms 1-4 of Section 3.
 *
 * Conventions shared by every entry point
 *  - Grids. d is 2 or 3; every N_a is odd (Section 2.1). A field on a grid of order N is d
 *    contiguous components, each an array N_1 x ... x N_d in C order (axis d contiguous);
 *    component a belongs to spatial axis a. Along every axis, storage index j holds the node
 *    x = m / N_a with signed index m = j for j <= (N_a - 1)/2 and m = j - N_a otherwise, so
 *    index 0 is the node x = 0 ("FFT-natural order"). Fourier coefficients use the same order.
 *  - Inner products and norms carry the 1/|N| weight of the Notation section.
 *  - Supported axis lengths: odd, 3 to 1023, every prime factor at most 31.
 *  - Pointers named *_dev are device pointers (cudaMalloc or torch tensors) on the device that
 *    was current at hom_create; all other array pointers are host pointers.
 *  - Work is issued on the stream passed to hom_create; every call that returns results to
 *    the host synchronises that stream before returning.
 *  - Every entry point returns a hom_status. On an error no output is written unless stated.
 *  - Ownership: hom_create copies the coefficient data; the caller keeps its buffers. The
 *    problem handle owns all device memory it allocates; hom_destroy frees it.
 *  - Elasticity (HOM_A_STIFFNESS; Section 1 names it among the "more involved applications"):
 *    fields are symmetric strain tensors with nc = d (d + 1) / 2 components in Mandel order
 *    (d = 2: e_11, e_22, sqrt2 e_12; d = 3: e_11, e_22, e_33, sqrt2 e_23, sqrt2 e_13,
 *    sqrt2 e_12), so the Frobenius product is the Euclidean product of the components; the
 *    projection G of eq. (discrete_proj) becomes the orthogonal projection onto compatible
 *    strains, Gamma^(k) e = (k q^T + q k^T)/|k|^2 - (k.e.k) k k^T/|k|^4 with q = e k, and
 *    (A_H E, E) the energy (C(E + e), E + e). Wherever this header says "d components" or
 *    "d doubles" for a field, E or a flux, read nc for such a problem.
 */
#ifndef HOM_H
#define HOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hom_problem hom_problem;

typedef enum {
  HOM_OK = 0,
  HOM_ERR_INVALID = 1,        /* bad argument (even N, d not 2/3, non-SPD phase, ...)     */
  HOM_ERR_OOM = 2,            /* device allocation failed                                  */
  HOM_ERR_UNSUPPORTED = 3,    /* e.g. Eyre-Milton with exact integration (Section 3.4)     */
  HOM_ERR_NOT_CONVERGED = 4,  /* iteration limit reached; results are still written        */
  HOM_ERR_CUDA = 5,           /* a CUDA call failed                                        */
  HOM_ERR_TIMEOUT = 6,        /* a device wait ran out: the FP32 strided pass on TMA-staged
                                 tiles waits for each tile's copy at most ~1 s of SM clock,
                                 then counts the failure and stops its CTA; hom_solve_end
                                 (and hom_solve) return this code when the count since the
                                 last check is not zero. The grid reductions take a
                                 completion ticket and never wait.                          */
  HOM_ERR_SCRATCH = 7         /* problem larger than the static scratch of hom_apply_static */
} hom_status;

/* Bytes of device memory reserved at load time, on every GPU that loads the library, for
 * hom_apply_static (held until the process exits). */
#define HOM_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

typedef enum { HOM_APPROX = 0 /* GaNi: A sampled at the nodes */,
               HOM_EXACT = 1  /* Ga: A_M on the double grid   */ } hom_integration;

typedef enum { HOM_RICHARDSON = 0, HOM_CG = 1, HOM_CHEBYSHEV = 2, HOM_EYRE_MILTON = 3 } hom_solver;

typedef enum { HOM_FP64 = 0 /* all arithmetic in FP64 */,
               HOM_FP32_REFINED = 1 /* FP32 operator inside FP64 iterative refinement */ } hom_precision;

typedef enum {
  HOM_A_PHASE = 0,   /* phase index per node (uint8 or uint16) + nphase x d x d SPD table   */
  HOM_A_SCALAR = 1,  /* one isotropic conductivity (double) per node                         */
  HOM_A_FOURIER = 2, /* exact integration only: isotropic coefficients A^(n), n in Z_M, as
                        interleaved complex doubles (re, im) in FFT-natural order on the
                        double grid M (eq. (Ga_exact_integration))                           */
  HOM_A_STIFFNESS = 3 /* linear elasticity (GaNi; FP64, or HOM_FP32_REFINED with CG or
                        Chebyshev inner solves in field form): phase index per node + nphase
                        symmetric positive definite stiffness matrices nc x nc in Mandel form,
                        nc = d (d + 1) / 2; see "Elasticity" below                          */
} hom_material_kind;

typedef struct {
  int kind;              /* hom_material_kind                                                */
  const void* data;      /* PHASE: |N| indices; SCALAR: |N| doubles; FOURIER: |M| complex    */
  int index_bytes;       /* PHASE: 1 (uint8) or 2 (uint16)                                    */
  const double* table;   /* PHASE: nphase row-major symmetric d x d tensors (host);
                            STIFFNESS: nphase row-major symmetric nc x nc Mandel matrices     */
  int nphase;            /* PHASE: table length                                               */
  int data_on_device;    /* 1 if data is a device pointer                                     */
  double cA, CA;         /* bounds of eq. (A); 0 = derive from the table / field. Required for
                            FOURIER (A_M itself may be indefinite, Section 4.1)              */
  int M[3];              /* FOURIER: odd double-grid order per axis, 0 = 2N - 1 (any odd
                            M >= 2N - 1 integrates the Ga bilinear form exactly)              */
} hom_material;

typedef enum { HOM_STOP_DEFAULT = 0, HOM_STOP_RESIDUAL = 1, HOM_STOP_INCREMENT = 2 } hom_stop;

typedef struct {
  int maxit;          /* iteration limit (0 = 100000)                                         */
  int fixed_iters;    /* > 0: run exactly this many iterations, no stopping test; with
                         HOM_FP32_REFINED one inner solve of exactly this many FP32 steps from
                         zero and its FP64 update (tol is then ignored)                     */
  int stop;           /* hom_stop. DEFAULT: residual ||b - C x|| <= tol ||b|| for Richardson,
                         CG and Chebyshev; increment ||x_m - x_{m-1}|| <= tol ||E|| for
                         Eyre-Milton (Algorithms 1-4 print the increment test for Richardson) */
  double cA, CA;      /* override of the spectral bounds used by Richardson, Chebyshev, EM    */
  double inner_tol;   /* HOM_FP32_REFINED: relative tolerance of each FP32 inner solve (0=1e-4)*/
                      /* HOM_FP32_REFINED uses maxit as the outer limit (0 = 50); only CG
                         and Chebyshev run as inner solvers                                 */
  int check_every;    /* host polls the device stopping flag every this many iterations (0=8) */
  int out_flags;      /* hom_out_flag bits for the corrector output of hom_solve, hom_solve_end
                         and hom_solve_current                                                */
  int inner_form;     /* HOM_FP32_REFINED (CG or Chebyshev): 0 = the FP32 inner solves run
                         Algorithm 2 or 3 in potential coordinates (x = grad u: one-component
                         vectors, operator D* A D, Laplacian preconditioner; the same iterates
                         in exact arithmetic) on 3-D grids whose axes all have specialised FP32
                         plans, else in field form; 1 = always in field form               */
} hom_opts;

/* Where and on which grid the solve returns the corrector e (field of hom_opts.out_flags). */
typedef enum {
  HOM_OUT_HOST = 1,   /* the corrector argument is a HOST pointer (any host memory; the field is
                         copied out before the call returns)                                  */
  HOM_OUT_NGRID = 2   /* exact integration: return the samples of the corrector on the nodes of
                         the N grid (d x |N| doubles) instead of its values on the solve grid M
                         (d x |M|). The Ga iterate is a trigonometric polynomial of order N
                         (Section 2.3), so its N-grid samples determine it; no effect for GaNi */
} hom_out_flag;

typedef struct {
  int iterations;     /* iterations of the (outer) solver                                      */
  int matvecs;        /* applications of the FFT-based operator                                */
  int inner_iterations;/* HOM_FP32_REFINED: total FP32 inner iterations                        */
  int converged;
  double residual;    /* last stopping quantity, relative (residual / ||b|| or increment / ||E||)*/
  double true_residual; /* ||b - C x|| / ||b|| recomputed at exit                              */
  double time_ms;     /* device time of the solve                                              */
} hom_stats;

typedef enum {
  HOM_OP_AFFINE = 0,  /* y = G A (E + x) = C x - b                 eq. (linsys)                */
  HOM_OP_LINEAR = 1,  /* y = G A x = C x                                                        */
  HOM_OP_PROJECT = 2, /* y = G x                                   eq. (discrete_proj)          */
  HOM_OP_EM = 3,      /* y = F^{-1}(I - 2 G^)F (A - omega I) x     Algorithm 4, omega = sqrt(cA CA)*/
  HOM_OP_FP32 = 16,   /* flag, or-ed into the above: apply the FP32 operator of a
                         HOM_FP32_REFINED problem (x rounded to FP32, y widened to FP64)     */
  HOM_OP_X_HOST = 32, /* flag: x is a HOST pointer                                             */
  HOM_OP_Y_HOST = 64  /* flag: y is a HOST pointer                                             */
} hom_op;

/* Create a problem on grid N (GaNi: the solve grid; Ga: the trigonometric order, the solve grid
 * is M). Validates the arguments, copies the coefficients to the device (Ga: assembles
 * A_M^k = sum_n omega_M^{kn} A^(n) with the library's inverse FFT, eq. (Ga_exact_integration)),
 * plans the odd-length FFTs and allocates the solver state (Section 3 storage) and one
 * half-spectrum work buffer. stream: a cudaStream_t or NULL for the legacy default stream.
 * Ga takes A^(n) directly (HOM_A_FOURIER) or an image: with HOM_A_PHASE (scalar tables only) or
 * HOM_A_SCALAR the coefficient is constant on the cell of side 1/N around each node, whose
 * coefficients are A^(n) = prod_a sinc(pi n_a / N_a) (F_N a)(n mod N) (the cell integral of
 * eq. (FT_def); the image's DFT F_N of eq. (DFT) runs on the device). Errors: HOM_ERR_INVALID,
 * HOM_ERR_OOM, HOM_ERR_CUDA, HOM_ERR_UNSUPPORTED (Ga of a tensor table); *out is set only on
 * HOM_OK. */
int hom_create(int d, const int* N, const hom_material* A, int integration, int precision,
               void* stream, hom_problem** out);

/* Solve-grid order (GaNi: N, Ga: M) into M_out[0..d-1]; number of nodes into *nodes. */
int hom_grid(const hom_problem* P, int* M_out, long long* nodes);

/* Spectral bounds c_A, C_A used by the solvers (eq. (A)). */
int hom_bounds(const hom_problem* P, double* cA, double* CA);

/* One application of the FFT-based operator (see hom_op) on fields x -> y (d x |grid| doubles
 * each; x may equal y). E (host, d doubles) is read by HOM_OP_AFFINE only.
 * x and y are device pointers unless flagged HOM_OP_X_HOST / HOM_OP_Y_HOST in op:
 *  - page-locked host memory (cudaHostAlloc, cudaHostRegister, torch pin_memory) is read and
 *    written by the pass kernels themselves through its device mapping (over the host link
 *    of the GPU, no staging copy); x is read once by the first pass and y written once by
 *    the last;
 *  - any other host memory is staged through one of the problem's device vectors with copies
 *    on the stream (those copies wait for the host).
 * With device pointers only, the call is enqueued on the problem's stream and does not
 * synchronise; with a host y it returns once y holds the result. During a solve session the
 * staging vector is the one the solvers leave free between steps. */
int hom_apply(hom_problem* P, int op, const double* E, const double* x_dev, double* y_dev);

/* Solve C x = b (eq. (linsys)) for macroscopic field E (host, d doubles) with the given solver
 * and tolerance, starting from x_0 = 0 (Eyre-Milton: x_0 = E). Writes, when non-NULL:
 * x_dev: the corrector e (Eyre-Milton: e = G x_m, Section 4.4), d x |grid| doubles on the
 * device (opts->out_flags: HOM_OUT_HOST for a host pointer, HOM_OUT_NGRID for the N-grid
 * samples of a Ga corrector, d x |N| doubles);
 * AH_EE: (A_H E, E) as the energy (A(E + e), E + e) on the solve grid (eqs. (GaNi),
 * (ev_bounds_Ga)); flux (d doubles): <A(E + e)>; stats. Eyre-Milton with HOM_EXACT returns
 * HOM_ERR_UNSUPPORTED (Section 3.4). Returns HOM_ERR_NOT_CONVERGED, with outputs written, when
 * the iteration limit stops the solve. Synchronises the stream. */
int hom_solve(hom_problem* P, const double* E, int solver, double tol, const hom_opts* opts,
              double* x_dev, double* AH_EE, double* flux, hom_stats* stats);

/* hom_solve in three steps, for callers that interleave work (benchmarks, schedulers):
 * begin validates like hom_solve, sets x_0 and enqueues the initial residual; iterate enqueues
 * up to `iterations` further steps (fewer once the limit is reached) without synchronising,
 * unless `done` is non-NULL, in which case it waits for the stream and reports whether the
 * solver has stopped; end waits, then writes the same outputs and status as hom_solve. A
 * problem holds one session at a time; begin discards an unfinished one. */
int hom_solve_begin(hom_problem* P, const double* E, int solver, double tol, const hom_opts* opts);
int hom_solve_iterate(hom_problem* P, int iterations, int* done);
int hom_solve_end(hom_problem* P, double* x_dev, double* AH_EE, double* flux, hom_stats* stats);

/* Per-iteration diagnostics of the current (or last) session: the quantities behind the
 * convergence studies of Section 4 (residual norms, 4.2; guaranteed upper bound, 4.3).
 *
 * hom_solve_history copies into the HOST array out (cap entries) the stopping quantity of
 * every iteration, in the grid norm ||a||^2 = (1/|N|) sum_k |a^k|^2 of Section 1:
 *   - CG and Chebyshev (Algorithms 2-3): ||r_m||, the recursively updated residual;
 *   - Eyre-Milton, and Richardson stopping on the increment (Algorithms 4, 1): ||x_m - x_{m-1}||;
 *   - Richardson stopping on the residual: ||C x_{m-1} - b|| as formed at the start of step m
 *     (the last entry belongs to the returned iterate);
 *   - HOM_FP32_REFINED: the FP64 residual ||b - C x|| after each outer update.
 * *count receives the number of entries recorded (at most 2^20 are kept; none beyond cap are
 * written); 0 before any solve. Synchronises the stream.
 *
 * hom_solve_current writes the current iterate (d x |M| doubles, device x_dev) of an active
 * session, as hom_solve_end would return it at this point: x_m for Richardson, CG and
 * Chebyshev, G x_m for Eyre-Milton (Section 4.4), the FP64 iterate of the last outer update in
 * HOM_FP32_REFINED mode. With hom_energy and hom_bound it gives the energy and the guaranteed
 * upper bound of every iterate (eq. (guar_upper_bound_m)). Synchronises the stream;
 * HOM_ERR_INVALID without an active session. */
int hom_solve_history(hom_problem* P, double* out, int cap, int* count);
int hom_solve_current(hom_problem* P, double* x_dev);

/* Non-conformity of the current iterate of an active session (Section 4.4), in the grid norm:
 * ||G x_m + E - x_m|| for Eyre-Milton (x_m approximates E + e) and ||G x_m - x_m|| for the
 * conforming solvers (round-off; Ga: G_{N,M}). Writes one double to the host pointer `value`;
 * synchronises the stream; HOM_ERR_INVALID without an active session. */
int hom_solve_nonconformity(hom_problem* P, double* value);

/* Snapshot and restore of an FP64 solve session (a build extension; the paper's solves run to
 * the end). A snapshot is everything the next hom_solve_iterate reads: the five solver vectors
 * (5 x d x |M| doubles), the device scalars (step coefficients, norms, iteration count, stop
 * flags, Richardson's buffer index), the recorded history and the host-side step counters.
 * Restoring it into an active session of a problem created the same way (same d, grid,
 * integration, coefficients and launch plan — results then agree bit for bit) whose session
 * was begun with the same E, solver, stopping rule and iteration limit continues the solve
 * exactly where the snapshot was taken; use: preempting a long solve (snapshot, end or
 * destroy, later create, begin and restore). Every call synchronises the stream.
 *
 * hom_solve_snapshot_size writes the bytes a snapshot of P's active session takes (a header,
 * the vectors and room for the whole history). hom_solve_snapshot writes the snapshot to the
 * host buffer host_buf of `bytes` bytes (at least that size, else HOM_ERR_INVALID).
 * hom_solve_restore reads one back; HOM_ERR_INVALID if it is not a snapshot, or was taken from
 * a session of another shape, solver, stopping rule, limit or E. A snapshot holds the
 * library's internal scalar layout: restore it with the same build of the library that wrote
 * it. The restoring session keeps its own polling interval and output flags.
 * HOM_FP32_REFINED sessions: HOM_ERR_UNSUPPORTED; no active session: HOM_ERR_INVALID. */
int hom_solve_snapshot_size(hom_problem* P, size_t* bytes);
int hom_solve_snapshot(hom_problem* P, void* host_buf, size_t bytes);
int hom_solve_restore(hom_problem* P, const void* host_buf, size_t bytes);

/* Energy (A(E + x), E + x) and flux <A(E + x)> of a device field x_dev on the solve grid
 * (x_dev may be NULL for x = 0, the Voigt value of Section 4.3). Synchronises the stream. */
int hom_energy(hom_problem* P, const double* E, const double* x_dev, double* energy, double* flux);

/* Prolongation R_{N,M} = I_M o I_N^{-1} (eq. (ev_bounds)): the trigonometric polynomial with
 * nodal values x_dev on the grid of `coarse` sampled on the solve grid of `fine`
 * (every M_a >= N_a, odd). Output y_dev: d x |M| doubles on the device. Vector fields only:
 * HOM_ERR_UNSUPPORTED for strain fields (elasticity). */
int hom_prolongate(hom_problem* coarse, hom_problem* fine, const double* x_dev, double* y_dev);

/* Guaranteed upper bound of eq. (ev_bounds_GaNi): U_E(R_{N,M}[E + x]) with x_dev a GaNi field
 * of problem `gani` and A_M of the exact-integration problem `ga` built for the same N.
 * Synchronises the stream. HOM_ERR_UNSUPPORTED for an elasticity problem (no exact
 * integration of stiffness). */
int hom_bound(hom_problem* gani, hom_problem* ga, const double* E, const double* x_dev,
              double* UE);

/* hom_apply_static: the GaNi operator of hom_apply for callers that cannot allocate device
 * memory. The paper has no counterpart; this entry point exists for integration only.
 *
 * Who needs it: a host application that owns every byte of device memory through its own
 * allocator or a fixed budget (and plugins running inside one), and latency-critical loops
 * that cannot pay for cudaMalloc/cudaFree, which may synchronise the device. hom_create
 * allocates; this call does not: it calls no cudaMalloc, cudaFree or allocating library
 * routine. Its work memory (half spectrum, twiddles, coefficient table) lives in one static
 * device array of HOM_STATIC_SCRATCH_BYTES that the library reserves when it is loaded.
 *
 * Arguments: d = 2 or 3, N (d odd orders, as hom_create), phase_dev a DEVICE array of |N|
 * phase indices (index_bytes 1 = uint8, 2 = uint16), table a HOST array of nphase row-major
 * SPD d x d tensors (symmetry and positive definiteness checked as in hom_create), op one of
 * hom_op (HOM_OP_EM uses omega = sqrt(c_A C_A) of the table), E (host, d doubles; read by
 * HOM_OP_AFFINE only), x_dev / y_dev device fields of d x |N| doubles in the layout of
 * hom_apply (distinct buffers), stream a cudaStream_t or NULL. The result equals hom_apply's
 * for the same problem (same plans, tables and kernels).
 * Precondition: every phase index is below nphase. The indices live on the device and are
 * not checked (hom_create reads them back and rejects them; this call does not); an index
 * out of range reads past the coefficient table and gives a wrong result.
 *
 * Limits and errors: the half spectrum (16 d |N| (N_d + 1) / (2 N_d) bytes) must fit in
 * HOM_STATIC_SCRATCH_BYTES minus 576 KiB (e.g. 135^3 with d = 3 fits, 243^3 does not); larger
 * problems return HOM_ERR_SCRATCH before any device work. Bad arguments: HOM_ERR_INVALID.
 *
 * Sharing: every call on a device uses the same scratch and leaves its contents behind;
 * nothing in it needs to start at zero (each call writes the twiddles, the table and every
 * spectrum entry before reading them). Calls whose work overlaps on the GPU (different
 * streams or threads without ordering) race on the scratch and give wrong results; issue them
 * on one stream or order them. Set-up: the first call on each device resolves the scratch
 * address (cudaGetSymbolAddress), uploads the DFT constants and sets the kernels'
 * shared-memory limits, so make that first call before any stream capture. Every call then
 * only enqueues kernels on `stream` (the twiddles and the table travel as kernel parameters,
 * not by host-to-device copies) and returns without waiting for the GPU. */
int hom_apply_static(int d, const int* N, const void* phase_dev, int index_bytes,
                     const double* table, int nphase, int op, const double* E,
                     const double* x_dev, double* y_dev, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched iterations and continuous batching (build extensions; the paper has one solve at
 * a time). Every request runs exactly the steps of a solo hom_solve with its own buffers,
 * device scalars and reduction partials, in a fixed reduction order, so its result is
 * bit-identical whether it runs alone or batched with others.
 * --------------------------------------------------------------------------------------- */

typedef struct hom_batch hom_batch;

/* Group `count` problems with an active session (hom_solve_begin) of the same solver,
 * precision, integration, grid and stream. The handles stay owned by the caller and must
 * outlive the batch. Errors: HOM_ERR_INVALID if they differ. */
int hom_batch_create(hom_problem* const* problems, int count, hom_batch** out);

/* Advance every member by `iterations` steps with one launch per pass for all members
 * (use_graph != 0: replay a captured CUDA graph of the batched step; ignored on the legacy
 * default stream, which cannot be captured). Members whose solver has
 * stopped skip their work on the device. all_done (nullable): synchronise and report whether
 * every member has stopped (for HOM_FP32_REFINED also runs the FP64 outer updates). Finish
 * each member with hom_solve_end. */
int hom_batch_iterate(hom_batch* B, int iterations, int use_graph, int* all_done);
void hom_batch_destroy(hom_batch* B);

typedef struct hom_server hom_server;

typedef struct {
  int d;
  int N[3];
  hom_material material;   /* host data only; copied at submit                              */
  int integration;
  int precision;
  double E[6];             /* nc entries: d, or d (d + 1) / 2 for a stiffness material      */
  int solver;
  double tol;
  hom_opts opts;
} hom_request;

typedef struct {
  long long id;
  int status;              /* hom_solve status of the request                              */
  double AH_EE;            /* (A_H E, E)                                                    */
  double flux[6];          /* nc entries                                                    */
  hom_stats stats;
  double latency_ms;       /* submit -> finished, host wall clock                           */
  double queue_ms;         /* submit -> admitted                                            */
} hom_result;

/* A continuous-batching solve server. Requests are admitted in arrival order while their
 * estimated device memory fits hbm_budget_bytes (at least one is always admitted), grouped into
 * buckets of equal grid, component count (conductivity or stiffness), integration, precision,
 * solver and inner form with up to max_batch slots each, and advanced together: one launch per
 * pass and bucket (captured CUDA graphs of the batched step), whatever the mix of arrival
 * times. Every bucket runs on a non-blocking stream of its own, so that buckets of different
 * grids overlap on the device; `stream` is not used. Finished requests free their slot and
 * memory at the step that detects them, and queued ones take their place. */
int hom_server_create(size_t hbm_budget_bytes, int max_batch, void* stream, hom_server** out);
/* Queue a request (the coefficient data is copied); *id identifies its result. */
int hom_server_submit(hom_server* S, const hom_request* req, long long* id);
/* Admit, advance every active request by `iterations` steps, retire finished ones, admit. */
int hom_server_step(hom_server* S, int iterations);
/* Move up to max finished results into out; *count = how many. */
int hom_server_poll(hom_server* S, hom_result* out, int max, int* count);
int hom_server_status(hom_server* S, int* active, int* queued, size_t* bytes_in_use);
void hom_server_destroy(hom_server* S);

/* Autotuner of the launch plan (build extension). For the grid of P it times `reps` operator
 * applications (after one warm-up) for every candidate register-radix limit (FP64: 9, 15; FP32:
 * 9, 15, 27), shared-memory tile budget per CTA (56, 80, 96, 110, 150, 200 KiB), thread count per CTA
 * of the runtime-radix passes (128, 256) and, in FP32, the two-line chain of the 3-D scalar
 * projection (on, off) where both column axes have specialised plans, re-plans P with the
 * fastest, and records the choice so that every later hom_create of the same grid, integration
 * support and precision in this process starts with it. Overwrites P's solver vectors (call it
 * before hom_solve_begin; HOM_ERR_INVALID during a session). report (nullable) receives the
 * choices and the time of one application. */
typedef struct {
  int rmax64, smem_kb64;
  double ms64;
  int rmax32, smem_kb32;   /* 0 unless P is HOM_FP32_REFINED */
  double ms32;
  int threads64, threads32;/* threads per CTA of the runtime-radix passes (128 or 256) */
  int two_line32;          /* 1: the FP32 3-D scalar projection keeps two spectrum lines
                              between its column passes (specialised plans on axes 0 and 1) */
} hom_tune_report;
int hom_autotune(hom_problem* P, int reps, hom_tune_report* report);

/* Re-plan P with a given launch plan (the fields of hom_tune_report: the FP64 ones, and for
 * HOM_FP32_REFINED the FP32 ones; times ignored), e.g. one that hom_autotune reported in an
 * earlier process, without timing candidates. Results change by rounding order at most.
 * HOM_ERR_INVALID for a plan outside the autotuner's candidates or during a session. */
int hom_set_plan(hom_problem* P, const hom_tune_report* plan);

/* Samples on the N grid (d x |N| doubles, device y_dev) of a field x_dev on the solve grid M of
 * an exact-integration problem whose spectrum lies in Z_N (every Ga iterate, Section 2.3):
 * F_M, the coefficients of Z_N, F_N^{-1} (eq. (DFT)); the inverse of hom_prolongate. For
 * GaNi problems (M = N) a copy. Enqueued on the problem's stream. */
int hom_restrict(hom_problem* P, const double* x_dev, double* y_dev);

/* Measurement utility (the paper has no counterpart): the FP64 rate of the current device.
 * Launches one untimed and one timed wave of chains of independent FP64 instructions on every
 * SM (kind 0: fused multiply-add, 2 flops each; kind 1: add, 1 flop), iters x 16 x 8 of them
 * per thread, timed with CUDA events on `stream`. Writes the timed launch's milliseconds and
 * its floating-point operations. Synchronises the stream. */
int hom_measure_fp64(int kind, int iters, void* stream, double* ms, double* ops);

/* Testing hook (the paper has no counterpart): make the n-th device allocation of the library
 * from now on fail (n = 0: the next one) as cudaMalloc does on a device without free memory;
 * the entry point that needed it frees what it had allocated and returns HOM_ERR_OOM. The
 * failure fires once; n < 0 disarms. Process-wide. */
int hom_debug_fail_alloc(int n);

/* Testing hook (the paper has no counterpart): on != 0 makes every TMA-staged strided pass
 * launched from now on wait for 16 bytes more than its tile copies deliver, so that each of
 * its waits runs out after ~1 s of SM clock; the CTAs stop, the copies that were issued land,
 * and the next hom_solve_end returns HOM_ERR_TIMEOUT. The results of such a solve are
 * meaningless; on = 0 restores normal operation. Process-wide. */
int hom_debug_tma_stall(int on);

/* Free everything the handle owns. NULL is accepted. */
void hom_destroy(hom_problem* P);

/* Static description of a status code. */
const char* hom_strerror(int status);

/* Number of kernels the library has launched in this process (a monotone counter). */
long long hom_kernel_launches(void);

/* Per-pass device timing for measurement: while enabled, every pass launch is bracketed by two
 * CUDA events on its stream. Enabling clears earlier records. Not thread-safe; intended for
 * benchmarks. Pass kinds: 0 pre-operator + forward DFT of the contiguous axis, 1 strided-axis
 * DFT, 2 axis-0 DFT with the projection, 3 inverse DFT of the contiguous axis + solver update,
 * 4 vector update / reduction kernels; the inner solves in potential coordinates
 * (HOM_FP32_REFINED, inner_form 0): 5 axis-0 iterate and direction update + inverse DFT,
 * 6 contiguous-axis inverse DFT + material + forward DFT, 7 axis-0 forward DFT + residual
 * update. */
int hom_profile_enable(int on);

/* Total milliseconds and launch counts per pass kind recorded since the last enable
 * (ms[k], launches[k] for k < nkinds <= 8). Waits for the recorded events. */
int hom_profile_read(double* ms, long long* launches, int nkinds);

#ifdef __cplusplus
}
#endif
#endif /* HOM_H */

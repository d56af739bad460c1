/*
 * bie2d.h -- C ABI of the GB300 (sm_103a) library for the resonance-free
 * second-kind integral equations of the 2D elastance and mobility problems
 * (Rachh & Greengard, "Integral equation methods for elastance and mobility
 * problems in two dimensions", arXiv:1507.05925).
 *
 * What is computed
 * ----------------
 * Elastance (Section 3): N conductors with boundaries Gamma_i carry prescribed
 * net charges q_i; the exterior potential u is harmonic, constant (= phi_i) on
 * each Gamma_i and decays at infinity (eqs. of Section 3.1).  With the uniform
 * incident density sigma_i = q_i/|Gamma_i| (eq. sigma) and u = S(mu + sigma)
 * (eq. TotRepresentation), mu solves the second-kind equation (eq. ModRep2)
 *     (1/2 I + K + L) mu = -(1/2 I + K) sigma,
 *     (K mu)(x) = int dG(x,y)/dn_x mu(y) ds_y,   G = -(1/2pi) log|x - y|,
 *     (L mu)(x) = int_{Gamma_i} mu ds   for x on Gamma_i.
 * Mobility (Section 4, viscosity 1): N rigid bodies with prescribed force F_i
 * and torque T_i (about the arc-length centroid x^c_i) move with (v_i, omega_i).
 * With rho_i = F_i/|Gamma_i| + T_i (x - x^c_i)^perp / W_i (eq. rho) and
 * u = S(mu + rho), mu solves (eq. ModRep2Stokes)
 *     (1/2 I + K + L) mu = -(1/2 I + K) rho,
 *     (K mu)_k(x) = n_l(x) int T_kml(x,y) mu_m(y) ds_y,  T_ijk = -(1/pi) r_i r_j r_k/|r|^4,
 *     (L mu)(x) = int_{Gamma_i} mu ds + (x - x^c_i)^perp int ((y - x^c_i)^perp, mu) ds.
 *
 * Discretisation: every boundary is sampled at theta_k = 2 pi k / n_i of a
 * smooth, counter-clockwise parametrisation; the Nystrom quadrature is the
 * periodic trapezoidal rule with weight w = |x'(theta)| 2 pi / n_i.  The
 * diagonal of K is its smooth limit -kappa/(4 pi) (Laplace) and
 * -(kappa/(2 pi)) tau tau^T (Stokes).  GMRES runs on the L2-rescaled unknowns
 * sqrt(w) mu (Section 6.1.1, rescaled linear system).
 *
 * Memory and ownership
 * --------------------
 * Every array argument is a plain pointer to HOST or DEVICE memory of the
 * context's device; the library tells them apart with cudaPointerGetAttributes.
 * Host inputs are copied in; when any output is host memory the call returns
 * only after the result has been written.  All device work is ordered on the
 * given stream (a cudaStream_t passed as void*, NULL = legacy default stream).
 * Input arrays are read-only and not retained after return; the caller owns
 * all input and output buffers.  The context owns its device workspace (the
 * Krylov basis, staged geometry, partial sums), which grows on demand up to
 * the cap given at creation.  A context is used by one host thread at a time.
 *
 * Errors
 * ------
 * Every entry point returns a status: 0 OK; > 0 a warning with a valid result;
 * < 0 an error, outputs untouched.  bie_last_error() gives a one-line message.
 */
#ifndef BIE2D_H
#define BIE2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BIE_OK 0
#define BIE_WARN_NONNEUTRAL 1    /* sum q != 0 (resp. sum F != 0): no decaying solution
                                    exists (Sections 3.1, 4.1, conservation conditions);
                                    the result is the free-space log-gauge field u = S(mu+sigma) */
#define BIE_WARN_NOT_CONVERGED 2 /* tolerance not reached within max_iter; info has the residual */
#define BIE_ERR_INVALID (-1)     /* bad argument: NULL pointer, N < 1, n_i < 8, non-monotone body_start,
                                    an array in device memory of a device other than the context's */
#define BIE_ERR_OUTSIDE (-2)     /* an interior evaluation point is not inside its body */
#define BIE_ERR_CUDA (-3)        /* a CUDA call failed (message in bie_last_error) */
#define BIE_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up (a grid barrier of the
                                    cooperative Arnoldi step waited about a second for a CTA that
                                    never arrived); the kernel returned, outputs are untouched and
                                    the context stays usable for the next call */
#define BIE_ERR_NOMEM (-5)       /* workspace needed exceeds the context's cap */

#define BIE_KIND_LAPLACE 0       /* elastance operator, scalar density [M] */
#define BIE_KIND_STOKES 1        /* mobility operator, node-interleaved density [2M] */

#define BIE_PREC_FP64 0          /* all arithmetic in IEEE double */
#define BIE_PREC_MIXED 1         /* pair sums in FP32 (FP32 accumulation per source tile);
                                    epilogue, Arnoldi, residuals and outputs in FP64 */
#define BIE_PREC_MIXED_FF 2      /* solves: as BIE_PREC_MIXED, but the refinement residual's pair
                                    sums run in float-float arithmetic on the FP32 pipes (about
                                    48 significant bits, positions split exactly into three
                                    floats) instead of FP64; apply_operator: float-float pair sums */

typedef struct bie_ctx bie_ctx;

/* Create a context bound to CUDA device `device`.  workspace_cap_bytes = 0
 * means no cap.  Returns BIE_OK and sets *ctx, or an error. */
int bie_create(bie_ctx** ctx, int device, size_t workspace_cap_bytes);

/* Release the context and its device workspace (NULL is ignored). */
void bie_destroy(bie_ctx* ctx);

/* Message of the last failure on this context ("" if none); owned by ctx. */
const char* bie_last_error(const bie_ctx* ctx);

/* Boundary geometry.  N bodies, M = body_start[N] nodes in total; body i owns
 * nodes [body_start[i], body_start[i+1]) sampled at theta_k = 2 pi k / n_i,
 * k = 0..n_i-1, n_i >= 8, counter-clockwise (Section 2: positively oriented
 * smooth closed curves).  All arrays float64 except body_start (int32). */
typedef struct {
  int32_t n_bodies;            /* N >= 1 */
  const int32_t* body_start;   /* [N+1], body_start[0] = 0, strictly increasing */
  const double* x;             /* [M] node x coordinate */
  const double* y;             /* [M] node y coordinate */
  const double* dx;            /* [M] dx/dtheta */
  const double* dy;            /* [M] dy/dtheta */
  const double* ddx;           /* [M] d2x/dtheta2 (curvature) */
  const double* ddy;           /* [M] d2y/dtheta2 */
  const double* interior_pt;   /* [2N] (x, y) per body, or NULL for the arc-length centroid;
                                  checked by a discrete winding number (BIE_ERR_OUTSIDE) */
} bie_geometry;

typedef struct {
  double tol;            /* stop when ||f - A nu|| <= tol ||f|| in the sqrt(w)-scaled 2-norm
                            (FP64 operator); default 1e-12 when <= 0 */
  int32_t max_iter;      /* cap on Krylov iterations over all cycles; default 500 when <= 0 */
  int32_t restart;       /* GMRES restart length m (1..200); default 50 when <= 0 */
  int32_t precision;     /* BIE_PREC_FP64 (GMRES in FP64), BIE_PREC_MIXED (FP64 iterative
                            refinement around FP32-pair-sum GMRES) or BIE_PREC_MIXED_FF
                            (the same refinement with float-float residual pair sums) */
  int32_t formulation;   /* 0: solve for the total density nu = mu + sigma with the
                            right-hand side L sigma (= q_i on Gamma_i), an identity of the
                            equivalence lemma (Section 3.5, 4.4); 1: the paper's form with
                            right-hand side -(1/2 I + K) sigma */
  int32_t max_refine;    /* mixed: cap on refinement steps; default 8 when <= 0 */
  double inner_tol;      /* mixed: relative tolerance of each FP32 inner solve; default 1e-6 */
  int32_t fmm_order;     /* 0: direct pair sums; p in 2..64: the pair sums are evaluated by the
                            quadtree FMM (FP64 expansions) with order p for residuals and FP64
                            GMRES, and order ceil(p/2) for the inner solves of the refinement;
                            -p (p in 2..64, mixed precisions only): direct FP32 pair sums for the
                            inner solves and the FMM of order p for the refinement's residuals and
                            the output sums (the reported residual is the FMM operator's, whose
                            relative error is about 1e-13 at p = 36) */
  int32_t precond;       /* right preconditioner of the GMRES iterations (the FP32 inner solves
                            of the mixed precisions, or the FP64 GMRES); 0: block Jacobi (one
                            block per body, the body's own diagonal block of the operator
                            GMRES iterates on, inverted in FP32; bodies over 640 unknowns, or
                            whose inversion meets a bad pivot, keep the identity), 1: none.
                            A right preconditioner leaves the residual GMRES minimises the
                            true one: it changes iteration counts, not the solution */
} bie_opts;

typedef struct {
  int32_t iters;               /* Krylov iterations (all cycles, all refinement steps) */
  int32_t refinements;         /* refinement steps taken (mixed), 0 for FP64 */
  int32_t matvecs_fp64;        /* FP64 operator applications */
  int32_t matvecs_fp32;        /* FP32-pair-sum operator applications */
  int32_t matvecs_ff;          /* float-float-pair-sum operator applications */
  double rel_residual;         /* final ||f - A nu|| / ||f|| in the sqrt(w)-scaled norm: with the
                                  FP64 operator, or (MIXED_FF without FMM) the residual updated
                                  with FP32 pair sums after the first true one plus the bound
                                  3 fp32_error sum ||A32 d|| of that update */
  double constraint_residual;  /* max_i |int_{Gamma_i} mu| (and Stokes moments) / max load */
  double net_load;             /* |sum_i q_i| or |sum_i F_i| */
  double fp32_error;           /* mixed: ||A32 x - A x|| / ||A x|| at the first refinement step,
                                  A32 the FP32-pair-sum operator of the inner solves and A the
                                  residual operator (FP64 or float-float); 0 for FP64 solves */
  int32_t precond_fallbacks;   /* block-Jacobi preconditioner: bodies whose diagonal block met a
                                  pivot that was not finite or tiny against the block's size during
                                  its inversion and that therefore keep the identity */
  int32_t graph_replay;        /* 1 when the GMRES iterations were replayed from a captured CUDA
                                  graph (a stream that can be captured), 0 when launched kernel by
                                  kernel (the legacy default stream, or pair-sum timing on) */
} bie_info;

/* Elastance solve (Section 3): charges q [N] -> conductor potentials phi [N].
 * density (nullable) receives the total density mu + sigma [M] (unscaled).
 * opts may be NULL (defaults), info may be NULL. */
int elastance_solve(bie_ctx* ctx, const bie_geometry* geom, const double* q, double* phi,
                    double* density, const bie_opts* opts, bie_info* info, void* stream);

/* Mobility solve (Section 4): loads FT [3N] = (Fx, Fy, T) per body ->
 * rigid motions UW [3N] = (vx, vy, omega) per body, omega about the body's
 * interior point (default the arc-length centroid x^c_i).  density (nullable)
 * receives mu + rho, node-interleaved [2M]. */
int mobility_solve(bie_ctx* ctx, const bie_geometry* geom, const double* FT, double* UW,
                   double* density, const bie_opts* opts, bie_info* info, void* stream);

/* Autotuning of the pair-sum grid (no counterpart in the paper).  Times one
 * application of the operator (pair sum + epilogue, CUDA events on the stream,
 * the fastest of five after two warm-ups) on this geometry for source-split
 * plans around the occupancy rule's -- uniform split counts, splits of whole
 * 256-source tiles, and (M >= 8192) two-level plans whose large chunks are
 * dispatched first and small chunks last -- and keeps the fastest for this
 * device and shape (M, kind, precision): later solves and operator applications
 * of that shape, in any context of the process, use it (the occupancy rule is
 * kept unless another plan is faster by 2%).  A different plan changes the
 * summation order, so results of that shape may change in rounding.
 * The FP32 and float-float Laplace pair sums have one more candidate, the
 * symmetric kernels (one CTA per unordered pair of 256-node tiles, each
 * difference, |r|^2 and reciprocal serving both directions of a pair; one
 * partial slot per tile), which are also the occupancy rule's plans once the
 * tile pairs fill the GPU four times over.
 * splits (nullable): on input 0 to search, a positive count to install a
 * uniform plan without timing (rounded to the counts the source chunking
 * allows), or a negative value to install the symmetric plan (Laplace with
 * BIE_PREC_MIXED or BIE_PREC_MIXED_FF only, else BIE_ERR_INVALID); on output
 * the number of splits of the plan kept, negated for the symmetric plan.  ms (nullable) receives its time (0 when
 * installed untimed).  Errors as for apply_operator. */
int bie_tune(bie_ctx* ctx, const bie_geometry* geom, int kind, int precision, int* splits, double* ms,
             void* stream);
/* FMM schedule tuning (no counterpart in the paper).  Times whole solves of
 * this geometry and load (kind 0 elastance, 1 mobility; opts->fmm_order = p in
 * 2..64 and a mixed precision) for candidate leaf populations (the leaf level
 * is the finest whose non-empty leaves hold at least 12, 24 or 48 nodes) and
 * inner-solve FMM orders (ceil(p/2) + {-4, -2, 0, 2, 4} within 2..p: a lower
 * order makes each inner iteration cheaper but may cost refinement steps), the
 * faster of two runs after a warm-up, and keeps the fastest candidate whose
 * solve converged for this device and shape (M, kind, p): later FMM solves and
 * apply_operator_fmm calls of that shape use it (the defaults 24 and
 * ceil(p/2) are kept unless another candidate is faster by 2%).  leaf_nodes,
 * inner_order and ms (nullable) receive the schedule kept and its solve time.
 * Errors as for the solves. */
int bie_tune_fmm(bie_ctx* ctx, const bie_geometry* geom, int kind, const double* load, const bie_opts* opts,
                 int* leaf_nodes, int* inner_order, double* ms, void* stream);

/* Forget every tuned split count and FMM schedule (back to the defaults). */
void bie_tune_clear(void);

/* Batched solves (no counterpart in the paper: a throughput path for many small
 * problems).  count independent problems of one kind -- geoms[p] with loads[p]
 * (q [N_p] or FT [3 N_p]) into outs[p] (phi [N_p] or UW [3 N_p]), host or device
 * arrays -- are solved together as one block-diagonal system: one set of
 * launches per GMRES iteration for all of them, every pair and output sum kept
 * inside its own problem.  Each problem has its own Krylov space (Hessenberg
 * matrix, rotations and stopping test); the problems advance in lockstep and a
 * problem that has converged stops taking part.  Each problem's right-hand side
 * is scaled to unit norm; every problem's own relative residual ends at most
 * opts->tol.  info (nullable) receives one bie_info per problem [count]: iters,
 * refinements and matvec counts are the batch's (lockstep iterations, those of
 * the slowest problem); rel_residual, constraint_residual and net_load are the
 * problem's own (mixed with float-float residual updates, rel_residual
 * includes their rounding bound).  status (nullable) receives each problem's
 * status [count] (BIE_OK, BIE_WARN_NONNEUTRAL, BIE_WARN_NOT_CONVERGED); the
 * return value is the worst of them, or an error for the whole batch.  Direct
 * pair sums only (fmm_order 0), no density output; interior points for all
 * problems or for none; 1 <= count <= 65535.  Errors: BIE_ERR_INVALID for a bad
 * argument in any problem (message names it). */
/* Batches of small problems -- every problem at most 1,024 nodes and 128
 * bodies, BIE_PREC_MIXED_FF, direct pair sums (fmm_order 0), restart <= 50 --
 * are solved by one persistent launch with one CTA per problem that runs the
 * problem's whole refinement (FP32-pair-sum GMRES on the correction equation
 * with the per-body weighted completion, no preconditioner; float-float
 * residuals; all reductions inside the CTA, in a fixed order), with no host
 * round trip until the end.  Each problem then stops at its own tolerance and
 * its bie_info counts (iters, refinements, matvecs) are its own.
 * bie_small_batch_path(0) sends such batches through the multi-launch path
 * instead (lockstep GMRES over the block-diagonal system); process-wide,
 * default on. */
void bie_small_batch_path(int enable);

int elastance_solve_batch(bie_ctx* ctx, int count, const bie_geometry* geoms, const double* const* q,
                          double* const* phi, const bie_opts* opts, bie_info* info, int* status, void* stream);
int mobility_solve_batch(bie_ctx* ctx, int count, const bie_geometry* geoms, const double* const* FT,
                         double* const* UW, const bie_opts* opts, bie_info* info, int* status, void* stream);

/* One application of the discrete second-kind operator (eqs. ModRep2,
 * ModRep2Stokes): out = (1/2 I + K + L) in, on unscaled densities.
 * kind = BIE_KIND_LAPLACE ([M] in/out) or BIE_KIND_STOKES ([2M], node-interleaved);
 * precision = BIE_PREC_FP64, BIE_PREC_MIXED (FP32 pair sum, FP64 epilogue) or
 * BIE_PREC_MIXED_FF (float-float pair sum, FP64 epilogue). */
int apply_operator(bie_ctx* ctx, const bie_geometry* geom, int kind, int precision,
                   const double* in, double* out, void* stream);

/* Operator application that allocates nothing (this entry point has no
 * counterpart in the paper; it serves callers that cannot allocate device
 * memory: code under a memory budget fixed in advance, inside a framework
 * that owns every device allocation through its own pool, or in a loop where
 * cudaMalloc/cudaFree, which may synchronise the device, are not allowed).
 * Same result as apply_operator (out = (1/2 I + K + L) in, unscaled), but
 * without a context: its scratch (staged geometry and pair-sum partials, about
 * 6 MB) is one fixed file-scope device array that every GPU loading this
 * library holds until the process exits.
 *   - Limits: M <= BIE_NOALLOC_MAX_NODES nodes and N <= BIE_NOALLOC_MAX_BODIES
 *     bodies; larger inputs return BIE_ERR_NOMEM and nothing runs.
 *   - Every array (geometry, in, out) must be device memory of the current
 *     device, or managed memory (BIE_ERR_INVALID otherwise).
 *   - Every call reads body_start back to the host and waits for the stream
 *     to finish that copy before it launches anything.
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress) with that device current: make that first call
 *     before any stream capture.
 *   - All calls on a device share the one scratch array: calls that overlap
 *     on the GPU (other streams, other host threads) race and corrupt each
 *     other's results; order them on one stream or serialise them.  Nothing
 *     in the scratch needs to start at zero: every call writes what it reads. */
#define BIE_NOALLOC_MAX_NODES 16384
#define BIE_NOALLOC_MAX_BODIES 2048
int apply_operator_noalloc(const bie_geometry* geom, int kind, int precision, const double* in,
                           double* out, void* stream);

/* Test hook for the bounded device waits (no counterpart in the paper).  Arms
 * a fault for the next fused Arnoldi step launched in this process: CTA
 * skip_cta of that launch leaves before its first grid barrier, and that
 * launch's barrier waits give up after `spins` polls of about 64 ns (instead of
 * about a second).  The other CTAs then record the timeout and return, and the
 * solve that made the launch returns BIE_ERR_TIMEOUT; nothing waits for ever.
 * A launch with fewer than skip_cta + 1 CTAs skips no CTA.  spins <= 0 disarms
 * the hook.  The hook is taken by one launch only. */
void bie_test_arm_barrier_timeout(int skip_cta, long long spins);

/* Test hook of the output sums' logarithm (no counterpart in the paper): for
 * device arrays x [n] and out [2n], out[i] = the table-driven FP64 logarithm
 * of x[i] that the output kernels use and out[n + i] = the CUDA library's
 * log(x[i]), so that a test can bound their difference.  Asynchronous on
 * `stream`; BIE_ERR_INVALID for NULL arrays or n < 0. */
int bie_test_log(const double* x, double* out, long long n, void* stream);

/* Test hook of the block-Jacobi safeguard (no counterpart in the paper): pivots
 * of later block factorisations count as bad when |p| < floor (default 1e-3 for
 * floor <= 0), so that a test can drive every body onto the identity block and
 * check bie_info.precond_fallbacks and the result. */
void bie_test_precond_pivot_floor(double floor);

/* apply_operator with the pair sums evaluated by the quadtree fast multipole
 * method in complex variables (Laplace: Re(nu F) with F the Cauchy sum of
 * q = w mu; Stokes: four Cauchy sums of q, conj(q) and q conj(z)), expansion
 * order p = order (2..64), FP64 expansions, direct near field.  Relative error
 * roughly 0.35^order of the operator's size. */
int apply_operator_fmm(bie_ctx* ctx, const bie_geometry* geom, int kind, int order, const double* in,
                       double* out, void* stream);

/* apply_operator_fmm in the arithmetic that a solve of the given precision
 * uses for FMM pair sums (the fast evaluation of the operator of Sections 3.4
 * and 4.3): BIE_PREC_FP64 as apply_operator_fmm; BIE_PREC_MIXED the inner
 * solves' operator (FP32 expansions of order p and an FP32 near field);
 * BIE_PREC_MIXED_FF the float-float refinement's residual operator (FP64
 * multipoles and local expansions, the multipole-to-local step in float-float
 * arithmetic, a float-float near field).  Arguments, ownership and errors as
 * for apply_operator_fmm; BIE_ERR_INVALID for another precision. */
int apply_operator_fmm_prec(bie_ctx* ctx, const bie_geometry* geom, int kind, int order, int precision,
                            const double* in, double* out, void* stream);

/* Device workspace (bytes) that elastance_solve (kind 0) or mobility_solve
 * (kind 1) needs for N bodies, M nodes and GMRES restart length `restart`
 * (0 = default): the Krylov basis, the staged geometry, the partial sums and
 * the staging of host inputs.  Requires a current CUDA device. */
size_t bie_workspace_bytes(int kind, int n_bodies, int n_nodes, int restart);

/* ---- Serving: continuous batching of solve requests ----
 * A server owns `workers` host threads, each with its own context and its own
 * non-blocking CUDA stream, so that the solves of concurrent requests overlap
 * on the device.  Requests wait in a queue and are admitted when a worker is
 * free and their workspace (bie_workspace_bytes) fits under hbm_cap_bytes
 * together with the requests in flight (0 = no cap); a request may pass an
 * earlier one that does not fit yet, but not more than 64 times.  Results do
 * not depend on what else is in flight: every kernel reduces in a fixed order
 * (unless batching is turned on, bie_server_batching). */
typedef struct bie_server bie_server;

typedef struct {
  int32_t kind;          /* BIE_KIND_LAPLACE -> elastance_solve, BIE_KIND_STOKES -> mobility_solve */
  bie_geometry geom;     /* arrays (host or device) must stay valid until the request completes */
  const double* load;    /* q [N] or FT [3N] */
  double* out;           /* phi [N] or UW [3N] */
  double* density;       /* nullable */
  bie_opts opts;         /* all zero = defaults */
} bie_request;

int bie_server_create(bie_server** srv, int device, int workers, size_t hbm_cap_bytes);
/* Queue a request (copied; its arrays are not).  Returns BIE_ERR_NOMEM at once
 * if the request alone exceeds the cap, BIE_ERR_INVALID for a malformed one. */
int bie_server_submit(bie_server* srv, const bie_request* req, int64_t* ticket);
/* Block until the request completes; returns its solve status and fills info
 * (nullable) and seconds (nullable) = time from submit to completion.  Each
 * ticket can be waited for once. */
int bie_server_wait(bie_server* srv, int64_t ticket, bie_info* info, double* seconds);
/* Batching of queued requests (off by default: max_batch 1).  A worker that
 * takes a request also takes up to max_batch - 1 queued requests of the same
 * kind, the same bie_opts and the same use of interior points (each of at most
 * max_request_nodes nodes, default 16,384; no density output, fmm_order 0;
 * 262,144 nodes a batch) and solves them together (elastance_solve_batch /
 * mobility_solve_batch); admission reserves the batch's workspace.  A batched
 * request's result agrees with its solo result to the solve tolerance, not
 * bitwise; with max_batch 1 results do not depend on what else is in flight.
 * 0 leaves a limit unchanged.  batches (nullable) receives the number of
 * batched solves (two or more requests) run so far. */
int bie_server_batching(bie_server* srv, int max_batch, int max_request_nodes, int64_t* batches);
/* Completed requests, workspace bytes of the requests now in flight, and the
 * largest such sum seen. */
int bie_server_stats(bie_server* srv, int64_t* completed, size_t* inflight_bytes, size_t* peak_inflight_bytes);
/* Finish the queued requests, stop the workers and free everything. */
void bie_server_destroy(bie_server* srv);

/* Measured arithmetic peaks of a device (no counterpart in the paper: the
 * denominators of the pair-sum rooflines).  Runs four short throughput kernels
 * on every SM of `device` (independent FMA / reciprocal chains, CUDA events,
 * the fastest of five runs) and writes out[4] = {FP32 FFMA TFLOP/s, FP32 packed
 * FFMA2 TFLOP/s (both counting an FMA as 2 flop), MUFU rcp.approx.f32 T op/s,
 * FP64 DFMA TFLOP/s}.  Takes about 20 ms; allocates 32 KB of device memory for
 * the duration.  BIE_ERR_CUDA if the device cannot run them. */
int bie_measure_alu_peaks(int device, double* out);

/* Kernel timing of the pair sums (the O(M^2) hot loop), for measurement.
 * counters[precision][kind] (precision 0 FP64, 1 FP32, 2 float-float): launches that did work and their summed device
 * time, taken with CUDA events recorded on the call's stream around each
 * pair-sum launch (launches skipped after GMRES convergence are not counted),
 * and the pair interactions they evaluated, M (M - 1) per launch.  enable = 1
 * clears the counters and starts timing, 0 stops it; out (nullable) receives
 * the counters so far.  kernel_launches counts every kernel this library
 * launched (on any stream) since timing was enabled. */
typedef struct {
  int64_t launches[3][2];
  double ms[3][2];
  double pairs[3][2];
  int64_t kernel_launches;
} bie_profile_counters;

int bie_profile(bie_ctx* ctx, int enable, bie_profile_counters* out);

#ifdef __cplusplus
}
#endif

#endif /* BIE2D_H */

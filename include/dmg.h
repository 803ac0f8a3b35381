/*
 * dmg.h -- C ABI of the B300-native differentiable multigrid solver (DMGS).
 *
 * Solves the steady diffusion-absorption problem of arXiv 2608.00760, Eq. 1,
 *
 *     -div(D grad u) + mu u = q          (mu: the absorption, lambda in the paper)
 *
 * on a structured vertex grid with zero Dirichlet boundary, discretised by
 * second-order central differences (7-point stencil; the coefficient on the
 * face between two vertices is the mean of their D values), by a multigrid
 * V-cycle with Red-Black Gauss-Seidel smoothing, full-weighting restriction
 * and trilinear prolongation (Sec. 2.2, Eqs. 5-7, Eq. 17), and exposes the
 * push-forward (JVP, Sec. 2.3) and pull-back (VJP, Sec. 2.4, Eq. 18) of the
 * solver. All arithmetic runs in CUDA kernels for sm_103a; the host code only
 * schedules them.
 *
 * Array convention (every double* below): nx*ny*nz float64 values, C order
 * [nz][ny][nx] (x fastest), covering ALL vertices including the boundary
 * planes. Each pointer may point to device memory or to host memory (pinned or
 * pageable); the library detects which and copies through its own buffers.
 * The caller owns every array; the library keeps no pointer to it after the
 * call returns. Values of q, w, dq and mu on boundary vertices are ignored
 * (Dirichlet); outputs u, du, qbar, mubar are written as 0 there, while Dbar
 * is defined on every vertex (boundary D enters the faces next to the
 * boundary).
 *
 * Batches: a context set up with batch = B > 1 holds B independent problems of
 * the same shape and parameters, each with its own D, mu and right-hand side
 * (the Monte Carlo samples of a variational-inference step, Sec. 2.5). Every
 * array above is then B such fields one after another, [B][nz][ny][nx]. Each
 * call runs all samples together, one launch per kernel and level, and each
 * sample stops at its own rtol: its result is bit for bit the result of the
 * same sample solved alone with batch = 1.
 *
 * Streams: every call takes a cudaStream_t (as void*; NULL = legacy default
 * stream) and orders all of its work on it. Calls return after the result has
 * been copied out (convergence tests need the residual norm on the host).
 * A context is not thread-safe: use one context per host thread/stream.
 *
 * Errors: every call returns a dmg_status; no call aborts the process.
 * dmg_last_error() gives a human-readable message for the last failure on a
 * context.
 */
#ifndef DMG_H
#define DMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmg_ctx dmg_ctx;

typedef enum {
    DMG_OK = 0,
    DMG_EINVAL = 1,   /* invalid argument: grid shape, NULL pointer, parameter range,
                         or a coarsest-level matrix that is not positive definite */
    DMG_ENOMEM = 2,   /* a device or pinned-host allocation failed (dmg_setup only) */
    DMG_ECUDA = 3,    /* a CUDA runtime call failed; see dmg_last_error */
    DMG_ENOCONV = 4,  /* rtol not reached within max_cycles; outputs hold the last
                         iterate and info->rel_residual its residual */
    DMG_ENAN = 5,     /* a residual norm was not finite (NaN/Inf in inputs) */
    DMG_ETIMEOUT = 6  /* reserved for bounded device waits (no kernel of the library
                         waits on a flag, so no call returns it) */
} dmg_status;

enum { DMG_FP64 = 0, DMG_MIXED = 1 };
enum { DMG_FACE_ARITHMETIC = 0, DMG_FACE_HARMONIC = 1 };
enum { DMG_COARSEN_FULL_WEIGHTING = 0, DMG_COARSEN_INJECTION = 1 };

/*
 * Solver parameters (dmg_default_params fills the defaults shown).
 *   nx, ny, nz    vertices per axis including both boundary vertices. The grid
 *                 is coarsened by 2 per axis (h_k = 2 h_{k-1}, Eq. 6) while
 *                 every axis has an odd count > 3; the coarsest level, solved
 *                 exactly, must have at most 512 interior unknowns.
 *                 2^n + 1 per axis (Sec. 2.2) always qualifies, and so does
 *                 c*2^n + 1 with small c (e.g. 257 x 257 x 129).
 *   h             finest spacing (> 0), equal on all axes.
 *   nu1, nu2      pre / post RB-GS sweeps per level (default 2, 2).
 *   symmetric     0: post-smoothing red->black like pre-smoothing (default);
 *                 1: post-smoothing black->red (then nu1 == nu2 gives a
 *                 symmetric V-cycle).
 *   max_cycles    cap on V-cycles (FP64) or refinement steps (mixed), default 100.
 *   rtol          stop when ||q - A u||_2 <= rtol ||q||_2 over interior vertices
 *                 (default 1e-10).
 *   fixed_cycles  0: iterate to rtol; m > 0: run exactly m V-cycles (the paper's
 *                 fixed-count mode, Sec. 2.4), FP64 only.
 *   precision     DMG_FP64 (default) or DMG_MIXED: FP32 inner V-cycles as the
 *                 correction of an FP64 defect-correction loop whose residual,
 *                 norms and update stay in FP64.
 *   face_mean     DMG_FACE_ARITHMETIC (default) or DMG_FACE_HARMONIC.
 *   coarsen       coarse coefficients: DMG_COARSEN_FULL_WEIGHTING (default; full
 *                 weighting inside, injection on the boundary) or INJECTION.
 *   inner_cycles  FP32 V-cycles per refinement step in mixed mode (default 3:
 *                 each step then gains ~3 decades, far above the FP32 floor).
 *   batch         independent problems in the context (default 1); needs
 *                 batch * nz <= 65535.
 *   autotune      0 (default): colour kernels use 32 x 8 thread blocks (FP64)
 *                 and, FP32 (two vertices per thread), 32 x 4 on wide levels,
 *                 16 x 8 or 8 x 16 on narrow ones; 1: dmg_setup
 *                 times the candidate block shapes of the half-sweep on every
 *                 grid level (FP64, and FP32 in mixed mode) and keeps the
 *                 fastest (one at least 3% faster than the default). Results are
 *                 reused within the process for the same device, precision,
 *                 grid, batch and face mean, and, if the environment variable
 *                 DMG_TUNE_CACHE names a file, read from and appended to it.
 *   split_prolong 0 (default): only the corrected values the first
 *                 post-smoothing half-sweep reads are formed: on 3D levels of
 *                 the FP32 V-cycle inside that half-sweep on levels of fewer
 *                 than 2^22 vertices (never stored), on larger ones and on 2D
 *                 levels by a correction of the other colour alone ahead of
 *                 a plain half-sweep (3D FP64 levels keep the full
 *                 prolongation, whose shared interpolations cost fewer FP64
 *                 operations); 1: the full
 *                 prolongation, then the half-sweeps. All give the same
 *                 results bit for bit.
 *   twin_adjoint  1 (default): dmg_solve_vjp runs the adjoint solve at the
 *                 same time as the forward one (it needs only w), on a second
 *                 context (the "twin": the same parameters and coefficient
 *                 hierarchy, its own iteration state and streams) that the
 *                 first dmg_solve_vjp call creates and dmg_set_coefficients
 *                 keeps in step; it doubles the device memory
 *                 (dmg_device_bytes counts it); when that memory cannot be
 *                 had the pair runs in one lane. The forward solve (the longer
 *                 one) is queued on a stream of the device's highest priority
 *                 and the adjoint one on a stream of the lowest, so that the
 *                 forward kernels take the SMs first where both lanes have
 *                 blocks waiting. Results are bit for bit those of running
 *                 the two solves one after the other. 0: one after the other
 *                 in this context.
 */
typedef struct {
    int nx, ny, nz;
    double h;
    int nu1, nu2;
    int symmetric;
    int max_cycles;
    double rtol;
    int fixed_cycles;
    int precision;
    int face_mean;
    int coarsen;
    int inner_cycles;
    int batch;
    int autotune;
    int split_prolong;
    int twin_adjoint;
} dmg_params;

#define DMG_HIST_LEN 64

/*
 * Per-call report. cycles: V-cycles run (FP64), or FP32 inner V-cycles (mixed);
 * outer: refinement steps (mixed; equals cycles in FP64); rel_residual: final
 * ||rhs - A x|| / ||rhs|| of the system solved; hist[c]: the relative residual
 * after cycle/step c (first DMG_HIST_LEN entries; not filled in fixed mode).
 * In a batch: the most cycles and steps of any sample, the largest final
 * relative residual, and in hist the largest over the samples that ran that
 * step (dmg_batch_info gives each sample's figures).
 */
typedef struct {
    int cycles;
    int outer;
    double rel_residual;
    double hist[DMG_HIST_LEN];
} dmg_info;

/* Fills *p with the defaults listed above (nx = ny = nz = 0, h = 0): the V(2,2)
   red-black schedule of Sec. 2.2 and the stopping rule of a 1e-10 relative
   residual. p may be NULL (no effect). */
void dmg_default_params(dmg_params *p);

/*
 * dmg_setup -- build the coefficient hierarchy (Sec. 2.2: L^k rediscretised
 * on every level h_k = 2 h_{k-1}) and every buffer the other calls use.
 *   D, mu   vertex fields of the diffusion coefficient (> 0) and absorption
 *           (>= 0), copied into the context; the caller may free them after.
 *   out     receives the new context (NULL on failure).
 * All device memory is allocated here; solve/jvp/vjp allocate nothing
 * (dmg_vjp_unrolled allocates its own work buffers on first use).
 * Returns DMG_EINVAL for an unsupported shape or parameter, or when the
 * coarsest matrix is not positive definite; DMG_ENOMEM when memory runs out.
 */
dmg_status dmg_setup(const dmg_params *p, const double *D, const double *mu, void *stream,
                     dmg_ctx **out);

/*
 * dmg_set_coefficients -- new coefficient fields for an existing context: the
 * hierarchy of Sec. 2.2 (D and mu coarsened level by level, the operator
 * rediscretised on every level, the coarsest matrix inverted) is rebuilt in
 * place for every sample, with the same kernels as dmg_setup and no
 * allocation; the context's buffers and captured graphs stay valid. This is
 * the per-iteration setup of a variational-inference loop, whose coefficients
 * are the quantities being inferred (Sec. 2.5).
 *   D, mu   as in dmg_setup ([batch][nz][ny][nx], device or host memory).
 * Synchronises the stream (to check the coarsest matrices). Returns
 * DMG_EINVAL for NULL arrays, while slots are running phases, or when a
 * coarsest matrix is not positive definite (the context then holds the new,
 * unusable coefficients until the next successful call).
 */
dmg_status dmg_set_coefficients(dmg_ctx *ctx, const double *D, const double *mu, void *stream);

/*
 * dmg_solve -- u = S(q) (Eq. 2): V-cycles from u = 0 until the relative
 * residual reaches rtol, or exactly fixed_cycles cycles. info may be NULL.
 * Returns DMG_ENOCONV (u still written) when max_cycles is reached first
 * (in a batch: by any sample).
 */
dmg_status dmg_solve(dmg_ctx *ctx, const double *q, double *u, dmg_info *info, void *stream);

/*
 * dmg_jvp -- push-forward (Sec. 2.3): du = S(dq - (dA) u), the tangent of
 * u(q, D, mu) in direction (dq, dD, dmu), where (dA) u is the derivative of
 * the discrete operator in (dD, dmu). With dD = dmu = NULL this is S applied
 * to dq, as the paper states for a solver linear in q; u is then not read
 * and may be NULL. dq may be NULL (zero). Same stopping rule as dmg_solve.
 */
dmg_status dmg_jvp(dmg_ctx *ctx, const double *u, const double *dq, const double *dD,
                   const double *dmu, double *du, dmg_info *info, void *stream);

/*
 * dmg_vjp -- pull-back (Sec. 2.4, Eq. 18) of the cotangent w:
 *   lambda = S^dagger w, qbar = lambda,
 *   mubar_p = -lambda_p u_p (interior), and
 *   Dbar_v = -(1/h^2) sum_{j nbr v} dDface(v,j)/dD_v (lambda_v-lambda_j)(u_v-u_j),
 * the gradients of <w, u> w.r.t. q, mu and D for the solution u of the forward
 * solve (the D and mu gradients are an extension the paper names as future
 * work in Sec. 4).
 *   cycles > 0  count-matched: exactly that many transposed V-cycles, the exact
 *               transpose of an m-cycle FP64 forward solve (the paper's second
 *               pull-back mode). Always FP64.
 *   cycles == 0 converged: iterate the adjoint to rtol (FP64 or mixed, as set up).
 * qbar, Dbar, mubar may each be NULL (skipped); u may be NULL when Dbar and
 * mubar are both NULL.
 */
dmg_status dmg_vjp(dmg_ctx *ctx, const double *u, const double *w, int cycles, double *qbar,
                   double *Dbar, double *mubar, dmg_info *info, void *stream);

/*
 * dmg_vjp_unrolled -- the exact gradient of <w, S_m(q; D, mu)> for the
 * fixed-count solver S_m: m FP64 V-cycles from u = 0 (Sec. 2.2), differentiated
 * through every iterate and through the coarsened coefficients of every level
 * (the pull-back of Sec. 2.4 extended to D and mu, which Sec. 4 names as future
 * work). It differs from dmg_vjp's gradient, which is that of the exact
 * solution, by the truncation of S_m; the two meet as m grows.
 *   m        cycles (>= 1); stride: iterates are recomputed from level-0
 *            checkpoints taken every `stride` cycles (0: ceil(sqrt(m))), so
 *            the memory grows with m / stride, not with m.
 *   u        receives S_m(q) (may be NULL); qbar = S_m^T w; Dbar, mubar the
 *            coefficient gradients (each may be NULL).
 * The forward cycles here use the grid kernels only (full defect, no
 * single-CTA tail), so S_m agrees with dmg_solve's fixed-cycle iterate to
 * rounding. Allocates its work buffers (about 2 (nu1 + nu2) + 9 fields per
 * level plus the checkpoints) on the first call and when m / stride grows.
 * Always FP64.
 */
dmg_status dmg_vjp_unrolled(dmg_ctx *ctx, const double *q, const double *w, int m, int stride,
                            double *u, double *qbar, double *Dbar, double *mubar, void *stream);

/*
 * The forward model of the paper's application (Sec. 2.5.3, Eq. response):
 *   L_e = R(q) = M(mu S(q)),
 * the absorbed energy density mu u on the voxels that lie at least `edge`
 * (a length, in the units of h; the paper masks 0.2 cm) from every face of
 * the grid. Along an axis of n vertices, voxel i is kept when
 * m <= i <= n-1-m, where m is the smallest integer with m h >= edge; the
 * other voxels of every output field are written as 0 (M^T M applied: the
 * data vector is the kept voxels in C order). edge = 0 keeps every voxel.
 *
 * dmg_response      -- Le = R(q); u (may be NULL) receives S(q).
 * dmg_response_jvp  -- dLe = M(mu du + dmu u), du = S(dq - (dA) u): the tangent
 *                      of R at (q, D, mu) in direction (dq, dD, dmu), any of
 *                      which may be NULL (zero); u = S(q) is required.
 * dmg_response_vjp  -- the pull-back of a cotangent rbar on Le:
 *                      w = mu M^T rbar, lambda = S^dagger w, qbar = lambda,
 *                      Dbar as in dmg_vjp with that lambda, and
 *                      mubar = -lambda u + u M^T rbar (the solve's term plus the
 *                      explicit factor mu). u = S(q) is needed for Dbar/mubar.
 * Stopping rule and statuses as in dmg_solve (the adjoint iterates to rtol).
 * Returns DMG_EINVAL for edge < 0 or not finite.
 */
dmg_status dmg_response(dmg_ctx *ctx, const double *q, double edge, double *Le, double *u,
                        dmg_info *info, void *stream);
dmg_status dmg_response_jvp(dmg_ctx *ctx, const double *u, const double *dq, const double *dD,
                            const double *dmu, double edge, double *dLe, dmg_info *info, void *stream);
dmg_status dmg_response_vjp(dmg_ctx *ctx, const double *u, const double *rbar, double edge,
                            double *qbar, double *Dbar, double *mubar, dmg_info *info, void *stream);

/*
 * dmg_solve_vjp -- dmg_solve followed by dmg_vjp (converged adjoint) in one
 * call: u = S(q) (Eq. 2), then (qbar, Dbar, mubar) of <w, u> through the
 * transposed V-cycle (Sec. 2.4, Eq. 18). Fusing the two calls has no
 * counterpart in the paper; it exists to run the two solves side by side and
 * to overlap host transfers. The adjoint solve needs w alone, so with
 * twin_adjoint = 1 (the default) it runs in the context's twin (created by the
 * first call: same parameters and hierarchy, own iteration state) on its own
 * stream and on a host thread the call starts and joins, while the forward
 * solve runs here; qbar is read out as soon as the adjoint solve ends. With
 * twin_adjoint = 0 the two solves run one after the other, w is uploaded
 * during the forward solve, u read out during the adjoint solve and qbar
 * during the gradient kernel. The forward solution stays on the device for
 * the gradients either way. The call waits for its work on `stream` before it
 * returns. Results are bit for bit those of the two calls. u, qbar, Dbar,
 * mubar may each be NULL; info_fwd / info_adj report the two iterations.
 * Returns the first non-OK status of the two (DMG_ENOCONV still writes every
 * output).
 */
dmg_status dmg_solve_vjp(dmg_ctx *ctx, const double *q, const double *w, double *u, double *qbar,
                         double *Dbar, double *mubar, dmg_info *info_fwd, dmg_info *info_adj,
                         void *stream);

/*
 * dmg_solve_vjp_many -- npairs fwd+VJP pairs in one call: for every i,
 * u[i] = S(q[i]) and the converged pull-back of w[i] (qbar[i], Dbar[i],
 * mubar[i]), as dmg_solve_vjp computes them (Sec. 2.3 forward, Sec. 2.4 /
 * Eq. 18 adjoint; streaming several pairs has no counterpart in the paper).
 * It exists for callers whose arrays live in host memory: pair i+1's q and w
 * are copied to the device while pair i iterates, and pair i's outputs are
 * copied back while pair i+1 iterates (an upload and a download stream, two
 * staging buffers each way), so the host transfers hide under the solves.
 *   q, w                 arrays of npairs pointers (none NULL), each a field as
 *                        in dmg_solve ([batch][nz][ny][nx], device or host).
 *   u, qbar, Dbar, mubar arrays of npairs output pointers, or NULL (that output
 *                        is skipped for every pair); an entry may be NULL.
 *   info_fwd, info_adj   arrays of npairs reports, or NULL.
 * With twin_adjoint = 1 each pair's adjoint solve runs in the twin beside its
 * forward solve (as in dmg_solve_vjp), and its gradients and read-out run on a
 * side stream while the next pair's solves start.
 * Host outputs are complete when the call returns (it synchronises). Results
 * are bit for bit those of dmg_solve_vjp on each pair. The first call
 * allocates the staging buffers (12 fields of the level-0 size) and two
 * streams, kept until dmg_destroy. Returns the first error (DMG_EINVAL,
 * DMG_ENAN, ...) and stops there, or DMG_ENOCONV if some pair reached
 * max_cycles (every output still written).
 */
dmg_status dmg_solve_vjp_many(dmg_ctx *ctx, int npairs, const double *const *q, const double *const *w,
                              double *const *u, double *const *qbar, double *const *Dbar,
                              double *const *mubar, dmg_info *info_fwd, dmg_info *info_adj, void *stream);

/*
 * dmg_residual -- out[2b] = ||q_b - A_b u_b||_2 and out[2b+1] = ||q_b||_2 over
 * interior vertices of every sample b, in FP64 (out is a host array of
 * 2 * batch doubles): the defect of Eqs. 13-14 on the finest level and the
 * norms of the stopping rule. q and u: caller arrays as in dmg_solve (device or
 * host, [batch][nz][ny][nx]). DMG_EINVAL for NULL arguments; synchronises the
 * stream before returning.
 */
dmg_status dmg_residual(dmg_ctx *ctx, const double *q, const double *u, double *out,
                        void *stream);

/*
 * dmg_batch_info -- per-sample report of the last solve/jvp/vjp on the context
 * (the Monte Carlo samples of a variational-inference step, Sec. 2.5, each with
 * its own coefficients; reporting per sample has no counterpart in the paper):
 * cycles[b] (V-cycles, or FP32 inner V-cycles in mixed mode) and rel[b] (final
 * relative residual; 0 for a zero right-hand side), host arrays of batch
 * entries each; either may be NULL. Before any such call every entry is 0.
 */
dmg_status dmg_batch_info(const dmg_ctx *ctx, int *cycles, double *rel);

/*
 * Slot-level interface (serving; no counterpart in the paper, whose solver
 * serves one call at a time). A context set up with batch = S is also a
 * pool of S slots for requests that arrive at different times: each slot holds
 * one request's coefficient hierarchy (kept resident while the request needs
 * it) and runs one phase at a time; every dmg_step_launch advances all running
 * slots together by one refinement step (mixed) or one V-cycle (FP64), one
 * launch per kernel and level for all of them, so requests admitted while
 * others run share the device (continuous batching). A slot's arithmetic is
 * that of its sample alone: its results are bit for bit those of
 * dmg_solve / dmg_jvp / dmg_vjp on a context of batch 1 with the same
 * parameters. Needs fixed_cycles == 0. While any slot is running a phase, the
 * whole-context calls (dmg_solve, dmg_jvp, dmg_vjp) return DMG_EINVAL.
 *
 * Phases:
 *   DMG_PHASE_FORWARD  u = S(q); a = q.
 *   DMG_PHASE_TANGENT  du = S(dq - (dA) u), u the slot's last forward solution;
 *                      a = dq, b = dD, c = dmu, each may be NULL (zero); b or c
 *                      needs a forward solution in the slot.
 *   DMG_PHASE_ADJOINT  lambda = S^dagger w (the converged adjoint, as dmg_vjp
 *                      with cycles = 0); a = w.
 * Arrays are one sample, [nz][ny][nx], device or host memory, read by the
 * calls' stream work (device arrays must stay valid until the next
 * dmg_step_finish has returned).
 */
enum { DMG_PHASE_FORWARD = 0, DMG_PHASE_TANGENT = 1, DMG_PHASE_ADJOINT = 2 };

/*
 * dmg_setup_pyramid -- a pool of slots for requests on a chain of grid sizes
 * that share their coarse levels (no counterpart in the paper). The grid
 * hierarchy of Sec. 2.2 for p's grid (nx, ny, nz) is the chain: level k has
 * (n - 1) / 2^k + 1 vertices per axis. slots_per_level[k] slots (k < nlevels)
 * take requests whose grid is level k, so a 257^3 pyramid serves 257^3,
 * 129^3, 65^3, ... requests together: slots are numbered level by level
 * (slots_per_level[0] slots of level 0 first), and every step launch runs one
 * V-cycle of all slots in which each level's kernels take every slot that
 * holds that level -- a 257^3 request's 65^3 level and a 65^3 request's finest
 * level in the same launch. Each slot's refinement (update, residual, norms)
 * runs on its own finest level, and its arithmetic is that of its request on a
 * context of its own grid: results are bit for bit those of
 * dmg_solve / dmg_jvp / dmg_vjp there.
 *   p          the chain's finest grid (nx, ny, nz), the vertex spacing h of
 *              every slot's own finest grid (requests of all sizes share h;
 *              a slot's coarser levels have 2h, 4h, ...), and the solver
 *              parameters (batch is ignored; fixed_cycles must be 0; 3D only).
 * Slots have no coefficients until dmg_slot_load; the slot calls take arrays
 * of the slot's own grid. Only the slot-level calls (and dmg_destroy,
 * dmg_device_bytes, dmg_levels, ...) accept a pyramid. Returns DMG_EINVAL for
 * bad counts, or when a level with slots would lie inside the single-block tail
 * of the small levels (its grid is too small; e.g. 17^3 in mixed precision).
 */
dmg_status dmg_setup_pyramid(const dmg_params *p, const int *slots_per_level, int nlevels, void *stream,
                             dmg_ctx **out);

/* dmg_slot_load -- rebuild the coefficient hierarchy of one slot from D, mu
   (asynchronous; a matrix that is not positive definite makes the slot's next
   phase end with DMG_EINVAL). The slot must not be running a phase. */
dmg_status dmg_slot_load(dmg_ctx *ctx, int slot, const double *D, const double *mu, void *stream);

/* dmg_slot_begin -- stage a phase into an idle slot (asynchronous); it starts
   iterating with the step after the next dmg_step_launch. */
dmg_status dmg_slot_begin(dmg_ctx *ctx, int slot, int phase, const double *a, const double *b,
                          const double *c, void *stream);

/* dmg_step_launch -- enqueue one step of every running slot and the read-back
   of their residual norms (asynchronous). Must be followed by dmg_step_finish. */
dmg_status dmg_step_launch(dmg_ctx *ctx, void *stream);

/* dmg_step_finish -- wait for the step, test every slot's relative residual
   against rtol (and max_cycles), and list in ended[0 .. *nended) the slots
   whose phase ended (ended may be NULL; it needs room for batch entries). A
   phase ends converged (DMG_OK), with DMG_ENOCONV, DMG_ENAN, or DMG_EINVAL for
   a slot whose load failed; dmg_slot_result gives the status. */
dmg_status dmg_step_finish(dmg_ctx *ctx, void *stream, int *ended, int *nended);

/* dmg_slot_result -- status (-1 while running), cycles and final relative
   residual of the slot's last phase; any output may be NULL. */
dmg_status dmg_slot_result(const dmg_ctx *ctx, int slot, int *status, int *cycles, double *rel);

/* dmg_slot_read -- copy results of an idle slot out (asynchronous on stream):
   u the slot's forward solution; x the last phase's solution (u, du or
   lambda = qbar); Dbar and mubar (after an adjoint phase) the coefficient
   gradients of <w, u> as in dmg_vjp. Any output may be NULL. */
dmg_status dmg_slot_read(dmg_ctx *ctx, int slot, double *u, double *x, double *Dbar, double *mubar,
                         void *stream);

/* Testing hook (fault injection on the host; no counterpart in the paper): the
   n-th device allocation made by the library from now on, process-wide, fails
   as if the device were out of memory (the call that made it returns
   DMG_ENOMEM and releases what it had allocated); n <= 0 turns it off. */
void dmg_debug_fail_alloc(long long n);

/* Testing hook, no counterpart in the paper: on = 1 makes every context of the
   process form D-bar and mu-bar with the per-vertex gradient kernel, which
   forms the differences of every face on both of its sides, instead of the
   tiled kernel that forms them once (arithmetic face mean); the two give the
   same bits. 0 (the default) turns it off. */
void dmg_debug_grad_per_vertex(int on);

/* Testing hook, no counterpart in the paper. Bounds-checked builds (compiled
   with -DDMG_BOUNDS_CHECK, the library's stand-in for a memory checker): the
   number of device accesses counted outside their arrays so far (every call
   also returns DMG_ECUDA when it added to it); -1 in normal builds. */
long long dmg_debug_oob_count(void);

/* Device memory held by the context, in bytes (for admission by memory budget;
   no counterpart in the paper). 0 for NULL. */
size_t dmg_device_bytes(const dmg_ctx *ctx);

/*
 * dmg_residual_static -- out[0] = ||q - A u||_2 and out[1] = ||q||_2 over
 * interior vertices in FP64, like dmg_residual, but with no context and
 * without allocating any device memory. The paper has no counterpart: this is
 * for callers that are not allowed to allocate device memory, e.g. code
 * running inside a host framework that owns the whole device pool through its
 * own allocator, or a latency-critical loop that cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree. Such callers cannot run
 * dmg_setup either, so this call works from their arrays alone.
 *   p          only nx, ny, nz, h and face_mean are read.
 *   D, mu, q, u  device memory of the current device, C order [nz][ny][nx],
 *              all vertices; boundary values of q and u are ignored.
 *   out        2 doubles, host or device memory.
 * The reduction's scratch is a fixed 4 MB file-scope device array that every
 * GPU which loads the library holds until the process exits. It bounds the
 * grid: (ny-2)*(nz-2) <= 262144 interior rows (513^3 fits); larger grids get
 * DMG_EINVAL with the reason in dmg_last_error(NULL).
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress and keeps it; make that first call before any stream
 * capture. The kept address does not survive cudaDeviceReset(): do not use
 * this entry point on a device after resetting it.
 * The call never reads or clears the thread's last CUDA error: an error the
 * caller left pending stays pending, and each CUDA call made here is checked
 * by its own return value.
 * All calls share the one array: calls that overlap on the GPU (other streams
 * or host threads) race and must be serialised by the caller. Each call writes
 * every scratch slot it reads, so no clearing is needed between calls. The
 * call returns after out is written (it synchronises the stream).
 */
dmg_status dmg_residual_static(const dmg_params *p, const double *D, const double *mu,
                               const double *q, const double *u, double *out, void *stream);

/* Frees every resource of the context (device and pinned host memory, streams,
   events, graphs). NULL is accepted. The context must not be in use on any
   stream; the call synchronises its own streams first. */
dmg_status dmg_destroy(dmg_ctx *ctx);

/* Static text for a status code. */
const char *dmg_strerror(dmg_status s);

/* Message of the last failure on ctx ("" if none). With ctx == NULL: the message
   of the last failed context-free call (dmg_setup, dmg_residual_static) on the
   calling thread. */
const char *dmg_last_error(const dmg_ctx *ctx);

/* Number of hierarchy levels and the vertex counts of level l (0 = finest): the
   grids of Sec. 2.2, h_l = 2^l h (Eq. 6). dmg_levels returns 0 for NULL;
   dmg_level_shape returns DMG_EINVAL for NULL or a level out of range. */
int dmg_levels(const dmg_ctx *ctx);
dmg_status dmg_level_shape(const dmg_ctx *ctx, int level, int *nx, int *ny, int *nz);

/* Thread-block shape (threads along the half-row, rows) of the colour kernels
   on a level, FP32 (fp32 != 0; threads take two vertices) or FP64: by default
   32 x 8 (FP64) and 32 x 4, 16 x 8 or 8 x 16 by the level's width (FP32), unless
   autotuned (no counterpart
   in the paper). DMG_EINVAL for NULL or a level out of range. */
dmg_status dmg_tile(const dmg_ctx *ctx, int level, int fp32, int *bx, int *by);

/*
 * Instrumentation (for benchmarks; no counterpart in the paper, which times
 * whole calls).
 * dmg_launch_count: kernels this context (and its twin) has launched so far.
 * dmg_profile_begin(ctx, kernel, level): from now on, bracket every launch of
 *   `kernel` (a DMG_KERNEL_* id) on `level` with CUDA events on its stream;
 *   at most `max_launches` event pairs are recorded. A run of consecutive
 *   half-sweeps (the nu1 or nu2 sweeps of one smoothing step) takes one event
 *   pair around the whole run and counts each of its launches, so the
 *   duration per launch includes the gaps between them but only 1/n of the
 *   cost of the event nodes themselves (a few microseconds each).
 * dmg_profile_end: waits for the recorded events and returns the number of
 *   recorded launches and their summed duration in milliseconds.
 * Profiling re-captures the context's graphs with event nodes in them; they
 * slow the calls down while it is on, so time the calls with it off.
 */
enum {
    DMG_KERNEL_SMOOTH = 0,     /* one RB-GS half-sweep (one colour) */
    DMG_KERNEL_RESTRICT = 1,   /* defect + full-weighting restriction */
    DMG_KERNEL_PROLONG = 2,    /* prolongation + correction (FP32 3D levels with
                                  post-smoothing: fused with the first post half-sweep,
                                  or, on levels of at least 2^22 vertices, the
                                  correction on the colour that half-sweep reads) */
    DMG_KERNEL_RESIDUAL = 3,   /* FP64 residual + norm */
    DMG_KERNEL_GRAD = 4,       /* coefficient gradients */
    DMG_KERNEL_TAIL = 5        /* the single-CTA V-cycle of the small levels; `level`
                                  is the first level it covers */
};
unsigned long long dmg_launch_count(const dmg_ctx *ctx);

/*
 * dmg_probe_fma -- measured FMA rate of the current device (instrumentation
 * for the roofline of the FP64 kernels; no counterpart in the paper): runs a
 * kernel of independent FMA chains on every SM (FP64 when fp64 != 0, else FP32)
 * on `stream`, times the third of three launches with CUDA events and writes
 * FMA instructions per second (one FMA = 2 flops) to *fma_per_s. Synchronises
 * the stream. DMG_EINVAL for a NULL output, DMG_ECUDA on a CUDA failure.
 */
dmg_status dmg_probe_fma(int fp64, double *fma_per_s, void *stream);
dmg_status dmg_profile_begin(dmg_ctx *ctx, int kernel, int level, int precision_fp32,
                             int max_launches);
dmg_status dmg_profile_end(dmg_ctx *ctx, long long *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* DMG_H */

/*
 * fdlb.h -- C ABI of the GB300 (sm_103a) IMEX finite-difference lattice
 * Boltzmann library (libfdlb.so).
 *
 * The library advances the two reduced distributions phi and chi of Kis &
 * Ambrus, "Implicit-Explicit Finite-Difference Lattice Boltzmann Model with
 * Varying Adiabatic Index":
 *   - phi = int f d(eta) d(zeta), chi = int (eta^2 + zeta^2) f d(eta) d(zeta)
 *     (Sec. II, Eq. galpha), so that D + K = 2/(gamma - 1) is free and gamma
 *     is any adiabatic index with K + D - d >= 0;
 *   - on the Gauss-Hermite product lattice of Qphi^d (phi) and Qchi^d (chi)
 *     momenta, roots of He_Q, weights absorbed (Sec. II);
 *   - with the Hermite-truncated equilibria of Eq. (gExpanded);
 *   - advection by the MP-9 monotonicity-preserving flux of Sec. IV, one 1-D
 *     sweep per axis, 5 ghost nodes per side (outlet: copies of the adjacent
 *     fluid node);
 *   - time stepping by the IMEX Runge-Kutta scheme of Eq. (IMEX) with the
 *     IMEX-SSP3(4,3,3) tableaux of Table I, every implicit BGK stage solved in
 *     closed form because collisions conserve n, u and T (Sec. III).
 *
 * Units: m = k_B = 1, momenta in units of the reference speed (Sec. II), so
 * the lattice momenta are the raw Hermite roots and n = rho, T = P/rho.
 *
 * State layout (host and device copies alike): one contiguous array
 *   F[P][ny][nx], x fastest (1-D: F[P][nx]), P = Qphi^d + Qchi^d;
 *   populations 0 .. Qphi^d-1 are phi_k, k = ky*Qphi + kx (1-D: kx);
 *   populations Qphi^d .. P-1 are chi_q, q = qy*Qchi + qx;
 *   momenta in ascending order along each axis.
 * Element type: double for both precisions.  An FDLB_MIXED context keeps
 * each population as an unevaluated sum of two binary32 numbers (high part
 * and the rounding residual below it) and converts to and from binary64 at
 * fdlb_get_state / fdlb_set_state.
 *
 * Ownership: the context owns every device buffer it allocates (cudaMalloc in
 * fdlb_create, freed by fdlb_destroy).  Callers own the arrays they pass in;
 * on_device = 0 means a host pointer (pageable or pinned), on_device = 1 a
 * device pointer of the context's device (e.g. a torch tensor's data_ptr()).
 * All work is enqueued on the context's CUDA stream; calls that return data
 * to host memory synchronise that stream before returning.
 *
 * Errors: every int-returning call returns FDLB_OK (0) or a negative code and
 * never aborts the process; fdlb_last_error() gives a one-line reason.
 * A context is not thread-safe: one caller thread at a time.
 */
#ifndef FDLB_H
#define FDLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDLB_OK 0
#define FDLB_EINVAL -1      /* bad argument: sizes, Q, gamma (K+D-d < 0), tau, dt, tableau */
#define FDLB_ECFL -2        /* |p| dt / ds > 1 for some lattice momentum (Sec. IV) */
#define FDLB_ENOMEM -3      /* device allocation failed */
#define FDLB_ECUDA -4       /* a CUDA runtime call failed (message in fdlb_last_error) */
#define FDLB_EUNSTABLE -5   /* a cell reached n <= 0, T <= 0 or a non-finite moment */
#define FDLB_ETIMEOUT -6    /* reserved: a bounded device wait gave up */

#define FDLB_FP64 0         /* populations stored and computed in binary64 */
#define FDLB_MIXED 1        /* binary32 storage and advection, binary64-accurate moments */

#define FDLB_BC_OUTLET 0    /* ghosts copy the adjacent fluid node (Sec. IV) */
#define FDLB_BC_PERIODIC 1  /* periodic images (conservation tests) */

typedef struct fdlb_ctx fdlb_ctx; /* opaque, library-owned */

/* Grid: d = 1 or 2 inhomogeneous axes, nx (and ny when d = 2) cells of the
 * domain [x0, x1] (x [y0, y1]); cell centres x_s = x0 + (s - 1/2) dx,
 * dx = (x1 - x0)/nx (Sec. IV).  bc is FDLB_BC_OUTLET or FDLB_BC_PERIODIC. */
typedef struct {
  int d;
  int64_t nx, ny;
  double x0, x1, y0, y1;
  int bc;
} fdlb_grid;

/* An r-stage IMEX tableau, row-major r x r: At (explicit, strictly lower),
 * A (implicit, lower), weights wt (explicit) and w (implicit).  The fused
 * kernels take any r = 4 tableau in which stage 1 is never advected
 * (At[i][0] = 0 for all i, wt[0] = 0) and stage 2 is not advected into
 * (At[1][*] = 0), as in Table I; others are rejected with FDLB_EINVAL. */
typedef struct {
  int r;
  double At[16], A[16], wt[4], w[4];
} fdlb_tableau;

/* Names for fdlb_named_tableau. */
#define FDLB_TABLEAU_IMEX_SSP3_433 0   /* Table I (the tableau NULL selects) */
#define FDLB_TABLEAU_EXPLICIT_SSPRK3 1 /* fully explicit comparator (Sec. VI) */

/* Fill *out with a named tableau (host only; no GPU needed).
 * FDLB_TABLEAU_EXPLICIT_SSPRK3 is the three-stage, third-order strong-
 * stability-preserving Runge-Kutta method of Shu and Osher applied to the
 * whole right-hand side, advection and collision alike (A = At, w = wt),
 * written as a 4-stage tableau whose first two stages are F^n itself so that
 * it runs through the same fused stage kernels.  With a_ii = 0 the closed-form
 * relaxation reduces to the explicit one: F^(i) = R_i and
 * dF^(i) = (dt/tau)(R_i - F_eq(R_i)).  Its real stability interval is about
 * dt/tau <= 2.5, so it needs dt of the order of tau; the paper's conclusion
 * (Sec. VI) quotes the IMEX step's dt/tau = 50 as the gain over such fully
 * explicit schemes.  Returns FDLB_EINVAL for an unknown name or NULL out. */
int fdlb_named_tableau(int which, fdlb_tableau* out);

/* Create a context and allocate its device buffers on the current device.
 *   grid       : see fdlb_grid (nx, ny >= 1; x1 > x0; y1 > y0 when d = 2)
 *   Qphi, Qchi : Gauss-Hermite orders per axis; supported pairs (8,8), (5,3),
 *                (3,3) in 1-D and 2-D
 *   gamma      : adiabatic index, D + K = 2/(gamma - 1), needs D + K >= d
 *   tau, dt    : BGK relaxation time (> 0) and time step (> 0);
 *                dt max|p| / dx <= 1 on every axis (Sec. IV CFL condition)
 *   tableau    : NULL for IMEX-SSP3(4,3,3) of Table I
 *   precision  : FDLB_FP64: populations stored and computed in binary64;
 *                FDLB_MIXED: populations stored as binary32 pairs (high
 *                part + residual); the MP-9 advection runs in binary32 on
 *                the high part shifted by a per-tile reference, the stage
 *                increments are kept as binary32 residuals relative to the
 *                high part; per-cell moment sums are binary64, so n, u, T
 *                (including the cancellation in T = (E - n u^2)/((D+K) n))
 *                are binary64, and the equilibrium factors are binary32
 *                pairs
 *   cuda_stream: cudaStream_t to enqueue on (NULL: the legacy default stream)
 *   out        : receives the context (NULL on failure)
 * The populations start at zero; call fdlb_init_riemann or fdlb_set_state. */
int fdlb_create(const fdlb_grid* grid, int Qphi, int Qchi, double gamma, double tau, double dt,
                const fdlb_tableau* tableau, int precision, void* cuda_stream, fdlb_ctx** out);

/* Set F to the discrete equilibrium (Eq. gExpanded) of piecewise-constant
 * Riemann data (Sec. V), n = rho, T = P/rho.
 *   1-D: nq = 2, states = {rho, u, P} left of xsplit, then right (cells with
 *        centre x >= xsplit take the right state);
 *   2-D: nq = 4, states = {rho, ux, uy, P} for quadrants 1 (x >= xsplit,
 *        y >= ysplit), 2 (x < xsplit, y >= ysplit), 3 (x < xsplit,
 *        y < ysplit) and 4 (x >= xsplit, y < ysplit).
 * The side of a cell is decided in cell units: cell i lies right of (above)
 * the membrane iff i + 1/2 >= s, s = (xsplit - x0) nx / (x1 - x0) computed in
 * binary64 in that order (likewise in y).  s is exact for a membrane at the
 * domain centre (s = nx/2), so with an odd cell count the middle cell, whose
 * centre lies on the membrane, takes the right (upper) state.
 * xsplit and ysplit must be finite (ysplit is ignored in 1-D).
 * states is a host array of nq*(d+2) doubles; rho > 0 and P > 0 required. */
int fdlb_init_riemann(fdlb_ctx* ctx, const double* states, int nq, double xsplit, double ysplit);

/* Advance nsteps >= 0 full IMEX steps on the context's stream: each step is
 * Eq. (IMEX) of Sec. III with the context's tableau (Table I by default), its
 * r stages each an explicit part R_i with the MP-9 advection of Sec. IV and
 * an implicit BGK relaxation solved in closed form (Sec. III).  The state is
 * advanced in place.  Returns FDLB_EUNSTABLE if any cell's moments became
 * invalid during these steps (checked once, after the last step, from a
 * device status word); the state then holds the invalid values. */
int fdlb_step(fdlb_ctx* ctx, int64_t nsteps);

/* fdlb_step that also reports, in stage_ms[0..2], the device time summed over
 * the nsteps steps of each fused kernel kind: stage 3, stage 4 and the final
 * stage (which also forms the next step's stage 2), from CUDA events recorded
 * on the context's stream between consecutive launches.  stage_ms is a host
 * array of 3 doubles. */
int fdlb_step_timed(fdlb_ctx* ctx, int64_t nsteps, double* stage_ms);

/* Moments of the current state (Eq. Moments_discrete): n, ux, uy (2-D only,
 * may be NULL in 1-D), T, each ncells = nx*ny doubles in [ny][nx] order.
 * on_device selects host or device destination pointers. */
int fdlb_moments(fdlb_ctx* ctx, double* n, double* ux, double* uy, double* T, int on_device);

/* Adjoint of fdlb_moments: the transpose of the Jacobian of (n, ux, uy, T)
 * with respect to the populations (Eq. Moments_discrete, with
 * T = (sum phi p^2 + sum chi - n u^2)/((D+K) n)), at the context's current
 * state.  nbar, uxbar, uybar, Tbar are device arrays of ncells doubles or
 * NULL (a zero adjoint; uybar is ignored in 1-D); Fbar (device, state layout,
 * binary64) is overwritten with sum_m mbar_m dm/dF.  The state is read only
 * when uxbar, uybar or Tbar is given (n is linear in F, so nbar alone needs no
 * state).  Binary64 single-problem contexts; FDLB_EINVAL otherwise.
 * Asynchronous on the context's stream. */
int fdlb_moments_adjoint(fdlb_ctx* ctx, const double* nbar, const double* uxbar,
                         const double* uybar, const double* Tbar, double* Fbar);

/* Copy the whole state F (layout above) out of / into the context.
 * fdlb_state_bytes gives the size: P * ncells * 8 (binary64 in both
 * precisions; FDLB_MIXED rounds each value to its binary32 pair on the way
 * in and returns the pair's sum, correctly rounded, on the way out). */
size_t fdlb_state_bytes(const fdlb_ctx* ctx);
int fdlb_get_state(fdlb_ctx* ctx, void* dst, int on_device);
int fdlb_set_state(fdlb_ctx* ctx, const void* src, int on_device);

/* Number of populations P and cells of the context (0 for NULL). */
int fdlb_npop(const fdlb_ctx* ctx);
int64_t fdlb_ncells(const fdlb_ctx* ctx);

/* Replace the context's stream (cudaStream_t, NULL = legacy default). */
int fdlb_set_stream(fdlb_ctx* ctx, void* cuda_stream);

/* Number of kernel launches fdlb_step makes per step (for launch accounting). */
int fdlb_launches_per_step(const fdlb_ctx* ctx);

/* ---- batches of independent 1-D problems ------------------------------------
 * One context holds nprob two-state problems of their own length and gamma
 * on the same domain [x0, x1], lattice, tau and dt.  Their cells are
 * concatenated: problem i owns cells [base_i, base_i + nx[i]) of the state
 * F[P][ncells], base_0 = 0, base_{i+1} = base_i + nx[i]; ghosts (Sec. IV)
 * copy each problem's own end cells.  Every stage runs all problems in one
 * launch of a persistent grid walking a work list of tiles, and fdlb_step
 * replays the steps from a captured CUDA graph.  fdlb_step, fdlb_step_timed,
 * fdlb_moments (n, u, T per concatenated cell), fdlb_get_state,
 * fdlb_set_state and fdlb_destroy work on batch contexts; fdlb_init_riemann
 * does not (use fdlb_batch_init_riemann).
 *   nx[nprob], gamma[nprob]: host arrays; nx >= 1, D+K-1 >= 0, CFL <= 1 each
 *   Qphi, Qchi: (8, 8) or (5, 3); precision: FDLB_FP64 or FDLB_MIXED */
int fdlb_create_batch(int nprob, const int64_t* nx, const double* gamma, double x0, double x1,
                      int Qphi, int Qchi, double tau, double dt, int precision, void* cuda_stream,
                      fdlb_ctx** out);

/* Equilibrium Riemann data of every problem of a batch: states is a host
 * array [nprob][2][3] of (rho, u, P) left and right, xsplit[nprob] the
 * membranes (NULL: the domain centres).  rho, P > 0. */
int fdlb_batch_init_riemann(fdlb_ctx* ctx, const double* states, const double* xsplit);

/* flags[nprob] (host): bit 0 set for each problem in which a cell reached
 * n <= 0, T <= 0 or a non-finite moment since the last initialisation.  The
 * problems do not interact, so the other members stay valid; fdlb_step
 * returns FDLB_EUNSTABLE as soon as any member is flagged. */
int fdlb_batch_status(fdlb_ctx* ctx, unsigned* flags);

/* base[nprob]: the first concatenated cell of each problem. */
int fdlb_batch_offsets(const fdlb_ctx* ctx, int64_t* base);

/* Autotuner of a batch context: times trial_steps steps of every tile shape
 * (cells per tile 127, 63, 255) and persistent-grid size (2, 4, 8, 16 CTAs
 * per SM) on the context's own problems, starting each trial from the
 * current state, restores the state and keeps the fastest shape.  The
 * chosen shape is returned in *variant_out and *ctas_per_sm_out (either may
 * be NULL).  Allocates one temporary state copy. */
int fdlb_autotune(fdlb_ctx* ctx, int trial_steps, int* variant_out, int* ctas_per_sm_out);

/* Set the batch tile shape directly (variant 0, 1, 2 = 127, 63, 255 cells). */
int fdlb_batch_set_tiling(fdlb_ctx* ctx, int variant, int ctas_per_sm);

/* ---- adjoint (1-D binary64 contexts with outlet ghosts and Table I) --------
 * Gradients of a loss of the final state with respect to the initial fields,
 * gamma and tau, by the discrete adjoint of the IMEX step: hand-written
 * kernels applying, in reverse stage order, the transposes of the step's
 * operations, with the MP limiter's choices frozen as the forward pass made
 * them (recomputed from the saved forward stage states), and the exact
 * Jacobian of the equilibria (Eq. gExpanded) with respect to the moments.
 * Checkpoints every `every` steps; each segment is recomputed once. */

/* F = discrete equilibrium of the per-cell fields n, u, T (device arrays of
 * ncells doubles). */
int fdlb_init_fields(fdlb_ctx* ctx, const double* n, const double* u, const double* T);

/* Adjoint of fdlb_init_fields: given Fbar (device, state layout), the fields'
 * adjoints nbar, ubar, Tbar (device arrays) and the contribution to
 * d/dgamma through chi^eq = (D+K-d) T phi^eq (*dgamma, host). */
int fdlb_init_fields_adjoint(fdlb_ctx* ctx, const double* Fbar, const double* n, const double* u,
                             const double* T, double* nbar, double* ubar, double* Tbar,
                             double* dgamma);

/* Advance nsteps from the current state, storing the state before steps
 * 0, every, 2 every, ... into ckpt (device, (nsteps/every + 1) states). */
int fdlb_forward_ckpt(fdlb_ctx* ctx, int64_t nsteps, int every, void* ckpt);

/* Reverse pass over the nsteps steps whose checkpoints fdlb_forward_ckpt
 * stored: Fbar (device, state layout) holds dLoss/dF(nsteps) on entry and
 * dLoss/dF(0) on return; dparams (host, 2) receives the step contributions
 * dLoss/dgamma and dLoss/dtau.  The context's state is left as it was.
 * Allocates its work space (8 every + 13 states: two segment buffers, so
 * that one segment's recompute overlaps the previous segment's adjoint on a
 * second stream the call creates and destroys) on first use; the context's
 * derived scratch arrays are rebuilt from its state before it returns. */
int fdlb_adjoint(fdlb_ctx* ctx, int64_t nsteps, int every, const void* ckpt, double* Fbar,
                 double* dparams);

/* The Gauss-Hermite rule of order Q (1 <= Q <= 16) the library uses for
 * weight exp(-p^2/2)/sqrt(2 pi): p[0..Q-1] the roots of He_Q in ascending
 * order, w[0..Q-1] = Q!/He_{Q+1}(p_k)^2 (Sec. II).  Host arrays; no GPU
 * needed.  Returns FDLB_EINVAL for Q out of range or NULL arrays. */
int fdlb_lattice_nodes(int Q, double* p, double* w);

/* Size of the static device scratch array used by fdlb_step_noalloc. */
#define FDLB_NOALLOC_SCRATCH_BYTES (64u << 20)

/* fdlb_step_noalloc -- advance a caller-owned binary64 state by nsteps IMEX
 * steps without allocating any memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, e.g. code
 * running inside another framework whose pool allocator owns all device
 * memory, or a real-time loop that may not take an allocation's latency and
 * device-wide synchronisation.
 *   grid, Qphi, Qchi, gamma, tau, dt, tableau : as for fdlb_create
 *   F          : device pointer to the state, layout F[P][ny][nx] (binary64),
 *                read as the initial state and overwritten with the result
 *   nsteps     : >= 0
 *   cuda_stream: stream to enqueue on (NULL: legacy default stream)
 * The intermediate arrays live in one static __device__ array of
 * FDLB_NOALLOC_SCRATCH_BYTES (64 MiB), which every GPU that loads the
 * library keeps until the process exits; problems with 5 * P * cells * 8 >
 * 64 MiB - 256 bytes are rejected with FDLB_EINVAL.  No cudaMalloc, cudaFree
 * or other allocating routine is called.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it; make that
 * first call before any stream capture.  All calls share the array: two
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and corrupt each other.  The call synchronises its stream to read the
 * status word; errors are reported through fdlb_last_error(NULL).  When it
 * returns FDLB_EUNSTABLE, F has already been overwritten and holds the state
 * in which the invalid moments appeared. */
int fdlb_step_noalloc(const fdlb_grid* grid, int Qphi, int Qchi, double gamma, double tau,
                      double dt, const fdlb_tableau* tableau, double* F, int64_t nsteps,
                      void* cuda_stream);

/* Measurement aid (no paper counterpart): the sustained binary64 fused
 * multiply-add rate of the current device, in DFMA per second, from a kernel
 * of 8 independent DFMA chains per thread on 8 CTAs of 256 threads per SM
 * (best of three timed launches after one warm-up, CUDA events on
 * cuda_stream).  This is the measured ceiling of the binary64 pipe that
 * bounds the binary64 stage kernels; an add or a multiply takes the same pipe
 * slot as an FMA.  *ms_out (may be NULL) receives the timed launch's ms.
 * Synchronises the stream; FDLB_ECUDA on a CUDA failure. */
int fdlb_measure_fp64_pipe(void* cuda_stream, double* dfma_per_s, double* ms_out);

/* Release the context and its device buffers (NULL is a no-op). */
void fdlb_destroy(fdlb_ctx* ctx);

/* One-line description of the last error on ctx (or of the last failed
 * fdlb_create when ctx is NULL); never NULL. */
const char* fdlb_last_error(const fdlb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FDLB_H */

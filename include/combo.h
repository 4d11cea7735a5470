/*
 * combo.h -- C ABI of libcombo.so: GB300 (sm_103a) FFT-based finite-strain
 * homogenization with composite boxels (ComBo).
 *
 * Method: Keshav, Fritzen, Kabel, "FFT-based homogenization at finite strains
 * using composite boxels (ComBo)", arXiv 2204.13624.
 *
 * The library solves the homogenization problem (HOM) of Sec. 2: for a
 * periodic RVE discretised by n1 x n2 x n3 voxels and a prescribed
 * macroscopic deformation gradient Fbar, find the compatible deformation
 * gradient field F with <F> = Fbar and Div P(F) = 0, and return the effective
 * first Piola-Kirchhoff stress Pbar = <P> (Eq. Pbar).  It uses the
 * finite-strain Lippmann-Schwinger equation of Sec. 3 (Eq. nonlinearLSE) with
 * the Green operator Gamma0 = Grad G0 Div (Eq. Gamma0) applied in Fourier
 * space.  Voxels cut by the material interface ("composite boxels") follow the
 * rank-one laminate law of Sec. 4 (Eqs. Fpm, tractionbalance, Peff:Seff),
 * solved per boxel by Newton-Raphson with selective back-projection
 * (Algorithms 1 and 2).  Both phases are compressible Neo-Hookean (Sec. 6.1).
 *
 * Conventions
 *   - 2-tensors are 9-vectors in row-major order F = [F11 F12 F13 F21 ... F33]
 *     (Sec. 1.5, Eq. vector:not).
 *   - Fields are component-major: X[c * V + v], V = n1 n2 n3, voxel index
 *     v = i + n1 (j + n2 k), i along x (fastest).
 *   - Phase codes: 0 = matrix ("-"), 1 = inclusion ("+"), 2 = composite boxel.
 *     Material index 0 is the matrix, 1 the inclusion.  A boxel's normal N
 *     points out of the inclusion into the matrix (Sec. 1.5, Sec. 5.1) and its
 *     c+ is the inclusion volume fraction.
 *
 * Ownership: the caller owns every pointer it passes.  combo_solve_begin and
 * combo_solve copy the problem during the call and keep no caller pointer.
 * Result arrays are caller-allocated and written before the call returns.
 *
 * Errors: every entry point returns COMBO_OK (0) or a negative COMBO_E_* code
 * and never throws; combo_last_error() gives a message for the calling
 * thread.  Numerical failures are status codes, never traps.
 */
#ifndef COMBO_H
#define COMBO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COMBO_OK 0
#define COMBO_E_INVALID_ARG (-1)
#define COMBO_E_OOM (-2)
#define COMBO_E_NOT_CONVERGED (-3)
#define COMBO_E_LAMINATE (-4)     /* a boxel Newton-Raphson did not converge */
#define COMBO_E_INADMISSIBLE (-5) /* det F <= 0 that step halving could not cure */
#define COMBO_E_NAN (-6)
#define COMBO_E_TIMEOUT (-7)
#define COMBO_E_CUDA (-8)
#define COMBO_E_CANCELLED (-9)

/* Where the pointers of a problem / result live. */
#define COMBO_MEM_HOST 0
#define COMBO_MEM_DEVICE 1

/* precision */
#define COMBO_FP64 0          /* every field and operator in FP64 */
#define COMBO_FP32_REFINED 1  /* FP32 Krylov iterations, FP64 residual, F, laminates, norms */
/* as COMBO_FP32_REFINED, but the residual G[P(F)] is evaluated in
   double-float arithmetic (pairs of FP32, 48-bit significand): the
   Neo-Hookean stress of the pure voxels (ln J included), the forward
   transforms and the projection; the inverse transforms, which only form the
   FP32 right-hand side of the Krylov solve, run in FP32.  The laminate
   Newton iterations run in double-float too, and an FP64 evaluation of the
   traction residual decides their convergence wherever the double-float
   rounding level does not lie clearly below the tolerance.  F stays FP64;
   the residual norms accumulate in FP64.  No counterpart in the paper: an
   arithmetic choice for GPUs whose FP64 rate is a small fraction of FP32. */
#define COMBO_FP32_REFINED_DF 2
/* kspace: discrete derivative of the Green operator */
#define COMBO_ROTATED 0  /* Willot's rotated scheme (HEX8R), Sec. 3 and Sec. 6.3 */
#define COMBO_SPECTRAL 1 /* Moulinec-Suquet trigonometric polynomials, Sec. 3 */
/* staggered grid (App. A, Eqs. forward_backward_difference, gradient_operator):
   F_aa = D_a^+ U_a, F_aB = D_B^- U_a (B != a), Div the adjoint of Grad; the
   nine components of a voxel's F sit at its centre (diagonal) and edge
   midpoints (off-diagonal), and the material law is applied to them as
   stored (the plain staggered scheme; no doubly-fine material grid).  Not
   available to combo_apply_G_noalloc. */
#define COMBO_STAGGERED 2
/* staggered grid with the doubly-fine material grid (App. A, Eq.
   constitutive_law): every voxel is cut into 8 sub-cells l in {0,1}^3; sub-cell
   l of cell c takes the diagonal of F at c and the off-diagonal pairs F_ab,
   F_ba at c + l_a e_a + l_b e_b (the edge nearest the sub-cell); the material
   of c is evaluated at each (a composite boxel: one laminate per sub-cell,
   each with its own jump vector), and the stress gathers
   P_aa[xi] = 1/8 sum_l S(xi, l)_aa, P_ab[xi] = 1/8 sum_l S(xi - l_a e_a - l_b e_b, l)_ab,
   the gradient of the sub-cell energy 1/8 sum_c sum_l W_c(F_sub(c, l)).  The
   operator is that of COMBO_STAGGERED.  All three solvers; Newton-CG applies
   the Hessian of the sub-cell energy (the sub-cell tangents applied to the
   direction assembled like F_sub and gathered like P).  combo_solve and
   combo_solve_begin only (not the batch, not combo_apply_G).
   combo_result.a_out holds the mean of a boxel's 8 sub-cell jumps;
   Pbar_phase averages over sub-cells. */
#define COMBO_STAGGERED_DFMG 3
/* solver */
#define COMBO_FIXED_POINT 0 /* basic scheme on the nonlinear LSE, Sec. 3 */
#define COMBO_NEWTON_CG 1   /* Newton with conjugate gradients on the linearised LSE, Sec. 3 */
/* nonlinear conjugate gradients on the nonlinear LSE (cited in Sec. 3; the
   paper gives no steps): Fletcher-Reeves directions d = -G[P]/mu0 + beta d,
   beta = ||G[P]||^2 / ||G[P]_prev||^2, and the basic scheme's step F += d.
   Like the fixed point: FP64, or the double-float residual form
   (COMBO_FP32_REFINED_DF). */
#define COMBO_NONLINEAR_CG 2

typedef struct combo_ctx combo_ctx;
typedef struct combo_solve_state combo_solve_state;

typedef struct {
    int32_t device;  /* CUDA device ordinal */
    void* stream;    /* cudaStream_t to launch on; NULL = the library creates its own */
} combo_ctx_opts;

/*
 * Problem statement (Sec. 2 HOM with the boxel data of Sec. 4).
 *   n[3]       grid n1, n2, n3; each 2^a 3^b, 2 <= n <= 1024, n1 even.
 *   l[3]       RVE edge lengths (voxel edge h_j = l_j / n_j; boxels may be
 *              non-equiaxed).
 *   phase      [V] phase codes (see above).
 *   n_boxels   number of composite boxels, == count of phase code 2.
 *   boxel_idx  [n_boxels] voxel index of each boxel, strictly increasing.
 *   boxel_N    [n_boxels][3] interface normal, normalised by the library;
 *              |N| < 1e-12 is rejected.
 *   boxel_c    [n_boxels] inclusion volume fraction c+ in (0, 1); boxels with
 *              c+ < c_min or c+ > 1 - c_min are evaluated as the pure phase.
 *   mu, lambda [2] Lame parameters of the Neo-Hookean phases; mu > 0,
 *              lambda > -2 mu / 3.
 *   Fbar       [9] macroscopic deformation gradient, det Fbar > 0.
 *   n_steps    load steps: Fbar_n = I + (n / n_steps)(Fbar - I), n = 1..n_steps.
 *   mem        COMBO_MEM_HOST or COMBO_MEM_DEVICE for phase/boxel_* pointers.
 */
typedef struct {
    int32_t n[3];
    double l[3];
    const uint8_t* phase;
    int64_t n_boxels;
    const int64_t* boxel_idx;
    const double* boxel_N;
    const double* boxel_c;
    double mu[2];
    double lambda[2];
    double Fbar[9];
    int32_t n_steps;
    int32_t mem;
} combo_problem;

/* theory: the kinematics and the phases' material law */
/* finite strain (default): compressible Neo-Hookean phases (Sec. 6.1), the
   laminate of Algorithm 1 and 2 in composite boxels (Sec. 4) */
#define COMBO_FINITE_STRAIN 0
/* infinitesimal strain (cheat sheet of the appendix, right column): the
   stored field F is I + H, H the displacement gradient; the phases are
   isotropic linear elastic, sigma = lam tr(eps) I + 2 mu eps, eps = sym(H),
   with the problem's (mu, lam); a composite boxel takes the closed form
   a = Delta^{-1} N . (C- - C+) : eps_box, Delta = N . (C+/c+ + C-/c-) . N,
   sigma_box = c+ sigma+ + c- sigma-, eps+- = eps_box +- sym(a (x) N)/c+-, and
   the tangent C_box = (c+ C+ + c- C-) - dC (N (x) Delta^{-1} (x) N) dC.  Pbar
   and P_out then hold sigma; det F is not constrained.  Not with
   COMBO_STAGGERED_DFMG. */
#define COMBO_INFINITESIMAL_STRAIN 1

/*
 * Solver options; combo_options_default() fills the defaults given here.
 *   precision        COMBO_FP64 (default), COMBO_FP32_REFINED or COMBO_FP32_REFINED_DF
 *                    (COMBO_FP32_REFINED with COMBO_NEWTON_CG only; with the fixed
 *                    point and nonlinear CG, COMBO_FP32_REFINED_DF evaluates every
 *                    residual -- law, doubly-fine sub-cell laws and gather, transforms --
 *                    in double-float arithmetic and keeps F in FP64; a doubly-fine boxel
 *                    sub-cell laminate converges to the tolerance or the double-float
 *                    rounding level)
 *   kspace           COMBO_ROTATED (default), COMBO_SPECTRAL, COMBO_STAGGERED or
 *                    COMBO_STAGGERED_DFMG
 *   solver           COMBO_NEWTON_CG (default), COMBO_FIXED_POINT or COMBO_NONLINEAR_CG
 *   tol              equilibrium tolerance on ||G[P]||_rms / |<P>|  (1e-8)
 *   max_iter         outer iterations per load step (200 Newton / 100000 fixed point)
 *   fixed_iterations > 0: run exactly this many outer iterations per load step
 *   cg_tol           CG stops at ||r|| <= cg_tol ||b||  (1e-3)
 *   cg_max_iter      (2000)
 *   cg_fixed_iterations > 0: exactly this many CG iterations per Newton step
 *   nr_tol_rel, nr_tol_abs  laminate NR stops at |f| <= rel (|P+N| + |P-N|) + abs mu_max (1e-12, 1e-14)
 *   nr_max_iter      laminate NR cap (50)
 *   c_min            boxel volume-fraction snap (1e-6)
 *   mu0              reference shear modulus of the fixed point; <= 0 picks
 *                    (min mu + max(lambda + 2 mu)) / 2
 *   theory           COMBO_FINITE_STRAIN (default) or COMBO_INFINITESIMAL_STRAIN
 *   wait_poll_cap    bound of every wait of the bulk-copy (TMA) kernels on their
 *                    copies: 0 (default) = 2^24 polls, k > 0 = k polls, -1 = none
 *                    (each such wait runs out at once; for testing the timeout
 *                    path).  A wait that runs out makes the kernel wait for its own
 *                    copies in flight, skip the rest of its work and raise
 *                    COMBO_E_TIMEOUT, which the call returns; the context stays
 *                    usable.
 */
typedef struct {
    int32_t precision;
    int32_t kspace;
    int32_t solver;
    double tol;
    int32_t max_iter;
    int32_t fixed_iterations;
    double cg_tol;
    int32_t cg_max_iter;
    int32_t cg_fixed_iterations;
    double nr_tol_rel;
    double nr_tol_abs;
    int32_t nr_max_iter;
    double c_min;
    double mu0;
    int32_t theory; /* COMBO_FINITE_STRAIN (default) or COMBO_INFINITESIMAL_STRAIN */
    int32_t wait_poll_cap;
} combo_options;

/*
 * Results, caller-allocated.  Pbar [n_steps][9] is required; every other
 * pointer may be NULL.
 *   F_out, P_out  [9][V] FP64 fields F and P(F), in `mem`: the converged
 *                 fields of the last step once the solve has finished, the
 *                 current iterate if combo_solve_finish ends it earlier.
 *   a_out         [n_boxels][3] laminate jump vectors, in `mem`.
 *   iters         [n_steps] outer (Newton / fixed-point) iterations.
 *   cg_iters      [n_steps] CG iterations.
 *   resid         [n_steps] final equilibrium residual.
 *   Pbar_phase    [n_steps][2][9] phase averages of P at each step's converged
 *                 state (Sec. 6.2): [0] the matrix, [1] the inclusion; pure
 *                 voxels add P and their volume to their phase, a composite
 *                 boxel adds c+- P+- (its laminate phase stresses at F+- =
 *                 F +- a (x) N / c+-) and c+- to each.  In `mem`.
 * Counters are totals over the solve.  steps_done is the number of load
 * steps completed (partial results are valid up to it on failure).
 */
typedef struct {
    double* Pbar;
    double* F_out;
    double* P_out;
    double* a_out;
    int32_t* iters;
    int32_t* cg_iters;
    double* resid;
    int32_t mem;
    int32_t steps_done;
    int64_t nr_iters;
    int64_t n_backproj;
    int64_t n_laminate_evals;
    int64_t n_operator; /* operator applications; voxel-iterations = n_operator * V */
    int64_t n_operator_fp64;
    double* Pbar_phase;
} combo_result;

/* Context: owns the device, the stream and the library's device memory.
 * Returns COMBO_E_CUDA if the device cannot be used.  opts may be NULL
 * (device 0, own stream). */
int combo_ctx_create(const combo_ctx_opts* opts, combo_ctx** out);
void combo_ctx_destroy(combo_ctx* ctx);

/* Message of the last error of the calling thread (never NULL). */
const char* combo_last_error(void);

void combo_options_default(combo_options* o);

/* Bytes of device memory one solve of this problem and options will hold. */
int64_t combo_solve_footprint(const combo_problem* p, const combo_options* o);

/* Full solve: copy the problem in, run every load step, write results. */
int combo_solve(combo_ctx* ctx, const combo_problem* p, const combo_options* o, combo_result* r);

/*
 * Batched solve (no counterpart in the paper, which solves one RVE at a time;
 * each problem is the problem of Sec. 2): n_problems independent problems,
 * each with its own grid n, cell size l, phase field, boxels, materials,
 * Fbar and number of load steps, solved together with the Newton-CG solver
 * (Sec. 3).  Problems of equal grid and cell size are stacked along z into
 * one grid (a class), so every kernel launch works on the pencils of all of
 * them (the x-passes give each problem its own blocks and reductions, the
 * z-passes transform each problem's segment).  With several classes, a class
 * of at least 2^20 stacked voxels runs its own tuned launch sequences on a
 * stream of its own, and for all smaller classes every pass of an operator
 * application -- laminate solves, x-forward, y, z with the Green operator, y
 * inverse, x-inverse -- is one persistent launch over a device table of
 * (class, block) work items on another stream, beside them; each CG chunk
 * replays from one captured CUDA graph with these streams as branches.  CG scalars, stopping tests, step
 * halving and results are per problem, and a problem that has converged is
 * masked out of the launches until the others finish the load step.
 *   problems[n_problems], results[n_problems]: as for combo_solve (each
 *   result's mem, pointers and sizes refer to its own problem).
 *   Errors: COMBO_E_INVALID_ARG for the fixed-point or nonlinear-CG solver
 *   with n_problems > 1; a failing problem fails the batch and the message
 *   names it.  n_problems == 1 is combo_solve.
 */
int combo_solve_batch(combo_ctx* ctx, int32_t n_problems, const combo_problem* problems, const combo_options* o,
                      combo_result* results);

/*
 * Incremental interface (used for timing and by the serving loop):
 *   begin    validates and copies the problem to the device, allocates the
 *            solve's fields; nothing runs yet.
 *   advance  runs until max_operator more operator applications are done
 *            (<= 0: no limit; the solver checks the count between its device
 *            loop chunks, so it may run a chunk past it) and returns COMBO_OK
 *            when every load step is done, COMBO_PENDING (1) when the limit
 *            stopped it, or an error.
 *   advance_newton  the same with min_operator > 0, but a reached limit
 *            stops the solve only between Newton steps (before the residual
 *            evaluation of the next Newton iteration, or between load steps),
 *            so every Newton step it starts -- residual, laminate solves, CG
 *            iterations and F update -- runs in full inside the call (used to
 *            time whole Newton steps); the fixed point and nonlinear CG stop
 *            between chunks as with advance.  COMBO_E_INVALID_ARG for
 *            min_operator <= 0.
 *   finish   writes the results; end frees the state.
 */
#define COMBO_PENDING 1
int combo_solve_begin(combo_ctx* ctx, const combo_problem* p, const combo_options* o, combo_solve_state** s);
int combo_solve_advance(combo_solve_state* s, int64_t max_operator);
int combo_solve_advance_newton(combo_solve_state* s, int64_t min_operator);
int combo_solve_finish(combo_solve_state* s, combo_result* r);
void combo_solve_end(combo_solve_state* s);

/*
 * Checkpoint / resume of a solve between load steps (no counterpart in the
 * paper; the load stepping F_n = I + (n/S)(Fbar - I) is this library's
 * reading).  The state that carries over a load step is F (FP64), the boxel
 * jump vectors (per sub-cell for COMBO_STAGGERED_DFMG), the step index, the
 * per-step results so far and the counters; everything else restarts with
 * each step.
 *   advance_steps  runs until k more load steps are done (COMBO_PENDING) or
 *                  the solve is (COMBO_OK); it stops between load steps.
 *   state_export   buf NULL: *bytes receives the size of the image; else
 *                  writes the host byte image into buf (*bytes its capacity
 *                  in, the size out).  Only between load steps (after
 *                  advance_steps, or when done); COMBO_E_INVALID_ARG else.
 *                  Single solves only (not batches).
 *   state_import   into a solve begun with the same problem and options and
 *                  not yet advanced; the header's grid, boxel count, step
 *                  count, k-space, solver, precision and theory must match
 *                  (COMBO_E_INVALID_ARG otherwise).  Advancing it then
 *                  continues with the next load step: with the same launch
 *                  shapes the result equals the uninterrupted solve's bit for
 *                  bit.  The image is host-endian and not a portable format.
 */
int combo_solve_advance_steps(combo_solve_state* s, int32_t k);
/* (the image: a header, the per-step results so far, then F [9][V] FP64 and
   the jump vectors [nb][3] FP64, and [nb][8][3] more on the doubly-fine grid) */
int combo_state_export(combo_solve_state* s, void* buf, int64_t* bytes);
int combo_state_import(combo_solve_state* s, const void* buf, int64_t bytes);

/*
 * Serving: a request loop for many solves of different grid sizes,
 * microstructures and load paths (no counterpart in the paper, which solves
 * one RVE at a time; each request is the problem of Sec. 2).
 *   combo_server_create  starts max_slots worker slots on ctx's device, each
 *                        with its own CUDA stream.  hbm_budget_bytes (<= 0:
 *                        85 % of the free device memory) bounds the sum of
 *                        the footprints (combo_solve_footprint) of the
 *                        running solves.  keep_fields: also keep F and P of
 *                        every finished request for combo_poll / combo_wait.
 *   combo_submit         validates and copies the problem (the caller may
 *                        free it on return) and queues it; returns a ticket.
 *                        A solve larger than the whole budget: COMBO_E_OOM.
 *   scheduling           a free slot admits the oldest queued request that
 *                        fits the memory left; each admitted solve keeps its
 *                        fields and iteration state on the device until it
 *                        finishes; requests arriving while others run are
 *                        admitted as slots and memory free up, and the running
 *                        solves' kernels overlap on the device.
 *   batching             with batch_max >= 2, a slot that admits a Newton-CG
 *                        request of at most batch_max_voxels voxels (<= 0:
 *                        96^3) also admits the queued requests with the same
 *                        grid, cell size and options, up to batch_max and the
 *                        memory left, and solves them together as one
 *                        combo_solve_batch (each request's result is the
 *                        result of its own solve); cancelling one request of a
 *                        running batch discards its result when the batch ends.
 *   combo_poll           COMBO_PENDING while running, else writes the result
 *                        (host pointers; the mem field is ignored) and
 *                        releases the ticket, returning the solve's status.
 *   combo_wait           same, blocking up to timeout_ms (< 0: forever);
 *                        COMBO_E_TIMEOUT if not finished in time (the ticket
 *                        stays valid).
 *   combo_cancel         a queued request finishes with COMBO_E_CANCELLED; a
 *                        running one stops at its next host round trip.
 *   combo_server_stats   counts and submit-to-completion latency percentiles
 *                        of the completed requests.
 *   combo_server_destroy cancels what is queued or running and joins the slots.
 */
typedef struct combo_server combo_server;
typedef struct {
    int32_t max_slots;
    int64_t hbm_budget_bytes;
    int32_t keep_fields;
    int32_t batch_max;         /* <= 1: no batching; else up to this many requests per batch */
    int64_t batch_max_voxels;  /* requests of at most this many voxels may be batched */
} combo_server_opts;
typedef struct {
    int64_t submitted, completed, failed, queued, running, peak_running;
    int64_t in_use_bytes, budget_bytes;
    double p50_seconds, p99_seconds, mean_seconds;
    int64_t batches, batched_requests; /* batches of >= 2 requests run, and their requests */
} combo_serving_stats;
int combo_server_create(combo_ctx* ctx, const combo_server_opts* opts, combo_server** out);
void combo_server_destroy(combo_server* s);
int combo_submit(combo_server* s, const combo_problem* p, const combo_options* o, int64_t* ticket);
int combo_poll(combo_server* s, int64_t ticket, combo_result* r);
int combo_wait(combo_server* s, int64_t ticket, int64_t timeout_ms, combo_result* r);
int combo_cancel(combo_server* s, int64_t ticket);
int combo_server_stats(combo_server* s, combo_serving_stats* st);

/*
 * Launch-shape autotuner (no counterpart in the paper).  The first Newton-CG
 * solve (or batch) of a grid -- sides, batch size, Krylov precision -- in
 * the process times the candidate launch shapes of each FP32 Krylov pass
 * (pass 0 tangent x-forward: 128- or 256-thread blocks, or in the nodal
 * form of the operator even shares of the (column, plane) pairs per block
 * or equal chunks of planes per column; 1 y-pass and 2 z-pass: two TMA
 * tile widths, of the scalar z-pass in the nodal form; 3 CG x-inverse: one
 * or two x-lines per group)
 * on the solve's own buffers before its first iteration, and every later
 * solve of that grid uses the fastest.  Shapes change no result beyond
 * floating-point summation order.
 *   combo_autotune_enable(0) keeps the default shapes for grids not yet tuned.
 *   combo_autotune_force(pass, cand) makes solves set up afterwards use
 *     candidate cand (0, 1) of pass (0..3), or the tuned one (cand = -1).
 *   combo_autotune_report writes one line per tuned grid (decisions and the
 *     time of 3 launches of each candidate) into buf (NUL-terminated, at most
 *     len bytes) and returns the full length.
 */
void combo_autotune_enable(int32_t enable);
int combo_autotune_force(int32_t pass, int32_t cand);
int64_t combo_autotune_report(char* buf, int64_t len);

/*
 * Evaluation forms of the rotated Green operator in the FP32 Newton-CG
 * Krylov passes (no counterpart in the paper; Sec. 3, the rotated scheme).
 * The rotated symbol k_J is, up to the unit factor i e^{i (theta_1 + theta_2
 * + theta_3) / 2}, the real kr_J of the symbol tables, and it is the Fourier
 * symbol of the HEX8R gradient D of a nodal field (edge differences along J
 * averaged over a voxel's 4 such edges, over h_J).  So G = D (D^T D)^+ D^T,
 * with D^T D the scalar |k|^2, and
 *   COMBO_KRYLOV_NINE          transforms all nine components of A : p both
 *                              ways and projects with k (k . X_i) / |k|^2;
 *   COMBO_KRYLOV_DISPLACEMENT  transforms nine components forward, leaves the
 *                              z-pass with the nodal field u_i = k^H X_i /
 *                              |k|^2 of each row and takes its gradient D u_i
 *                              in real space (three inverse transforms);
 *   COMBO_KRYLOV_NODAL         also assembles the nodal forces f_i = D^T (A :
 *                              p)_i in real space in the tangent pass (three
 *                              forward transforms, the z-pass divides by
 *                              |kr|^2); the direction p alternates between
 *                              two buffers (with a voxel map: 40 bytes
 *                              more per voxel).
 * Each is an evaluation order of the same operator: results agree up to FP32
 * rounding.  The reduced forms apply to single and stacked solves (and the
 * own-launch classes of batches over several grids) with the rotated scheme,
 * FP32 Krylov words, the TMA y- and z-passes (sides 48 ... 512 with
 * compile-time plans) and n1 = 128, 256 or 512 with n2 a multiple of 4;
 * other solves take the most reduced form that applies.
 *   combo_krylov_form(form) sets the most reduced form that solves set up
 *     afterwards may use (default COMBO_KRYLOV_NODAL); COMBO_E_INVALID_ARG
 *     outside 0..2.  Process-wide.
 */
#define COMBO_KRYLOV_NINE 0
#define COMBO_KRYLOV_DISPLACEMENT 1
#define COMBO_KRYLOV_NODAL 2
int combo_krylov_form(int32_t form);

/*
 * Per-kernel timing of a solve (instrumentation, no effect on results).
 *   combo_solve_profile(s, 1) resets the counters and records a CUDA event
 *   pair around every kernel launch of the solve on its stream; 0 stops.
 *   combo_solve_profile_read fills, for up to max_classes launch classes,
 *   names (32 chars each, may be NULL), total milliseconds and launch counts,
 *   and returns the number of classes.  Launch counts are kept also while
 *   timing is off.
 */
int combo_solve_profile(combo_solve_state* s, int32_t enable);
int combo_solve_profile_read(combo_solve_state* s, int32_t max_classes, char* names, double* ms,
                             int64_t* launches);

/*
 * Unit-level entry points (same kernels as the solve).
 *
 * combo_apply_G: Y = G[X] = mu0 Gamma0[X] (Eq. Gamma0 with C0 = mu0 I),
 *   X, Y [9][V] FP64 in `mem`; precision selects the FFT arithmetic (FP64,
 *   FP32, double-float);
 *   *sumsq receives sum_x |Y(x)|^2.
 * combo_constitutive: P[9][V] (FP64) of the field F[9][V] (FP64): pure
 *   voxels Neo-Hookean (Sec. 6.1), boxels the laminate (Algorithms 1-2)
 *   started from a_io[n_boxels][3] (updated in place); o->kspace and
 *   o->theory select the doubly-fine law and the infinitesimal-strain law,
 *   the arithmetic is FP64.  All in `mem`.
 */
int combo_apply_G(combo_ctx* ctx, const int32_t n[3], const double l[3], int32_t kspace, int32_t precision,
                  const double* X, double* Y, double* sumsq, int32_t mem);
int combo_constitutive(combo_ctx* ctx, const combo_problem* p, const combo_options* o, const double* F,
                       double* a_io, double* P, int32_t mem);

/*
 * Unit-level entry points, evaluated on the device by the solver's own code
 * (host arguments; for tests of the material routines in isolation):
 * combo_neohooke_eval: P(F) (Sec. 6.1, P = mu F + (lam ln J - mu) F^{-T}) and,
 *   if A is not NULL, the tangent A[9*(3i+J) + 3k+L] = dP_iJ/dF_kL; F, P
 *   row-major 3x3.  COMBO_E_INADMISSIBLE if det F <= 0.
 * combo_laminate_eval: one composite boxel (Sec. 4, Algorithms 1 and 2, FP64,
 *   NR tolerance 1e-12 relative / 1e-14 absolute, at most 50 iterations):
 *   F the boxel's F, N its normal (normalised here), c = c+ in (0, 1),
 *   mat = {mu-, lam-, mu+, lam+}; a_io the jump vector (warm start in,
 *   converged out); P = c+ P+ + c- P-; A (or NULL) the boxel tangent
 *   (Eq. Peff:Seff); *iters (or NULL) the Newton iterations.
 *   COMBO_E_LAMINATE / COMBO_E_INADMISSIBLE when the solve fails.
 */
int combo_neohooke_eval(combo_ctx* ctx, const double F[9], double mu, double lam, double P[9], double A[81]);
int combo_laminate_eval(combo_ctx* ctx, const double F[9], const double N[3], double c, const double mat[4],
                        double a_io[3], double P[9], double A[81], int32_t* iters);

/*
 * combo_df_log: the double-float natural logarithm that the double-float
 * forms use for ln J (series of 2 atanh((m - 1)/(m + 1)) after a power-of-two
 * range reduction), exposed so that its accuracy can be tested:
 * y[i] = ln x[i] evaluated in double-float and returned as FP64.  x, y host
 * arrays of n >= 0 doubles; every x[i] must be positive and within the
 * normal FP32 range (COMBO_E_INVALID_ARG otherwise, nothing computed).
 */
int combo_df_log(combo_ctx* ctx, const double* x, double* y, int64_t n);

/*
 * combo_arith_rates: the device's FMA throughput (no counterpart in the
 * paper; the denominators of the rooflines of the kernels bound by
 * arithmetic rather than memory, such as the laminate solve).  Launches
 * 2048 threads per SM, each running 8 independent chains of dependent FMAs
 * (no memory traffic), on the context's stream, timed with CUDA events
 * (best of three after a warm-up, a few ms each).  tflops: host array of 2
 * doubles, written with the FP64 and FP32 rates in TFLOP/s (an FMA counts
 * as 2 FLOPs).  Synchronises the context's stream.
 */
int combo_arith_rates(combo_ctx* ctx, double* tflops);

/*
 * combo_coarse_grain: composite boxels from a binary fine image (Sec. 5).
 *
 * The fine image of n1 x n2 x n3 voxels (edges h) is cut into coarse voxels
 * of b1 x b2 x b3 fine voxels (b_j divides n_j), nc_j = n_j / b_j.  A coarse
 * voxel whose fine voxels are all matrix gets phase 0, all inclusion phase 1,
 * both phases phase 2: a composite boxel with c+ = (its inclusion voxels) /
 * (b1 b2 b3) and an interface normal N.
 *
 * method COMBO_NORMAL_LAPLACE (Sec. 5.1-5.2): weights w = |S * chi| of the
 *   periodic discrete Laplacian whose axis-i second difference is scaled by
 *   r_i = h_j h_k / h_i; N is the eigenvector of the smallest eigenvalue of
 *   the boxel's second moment M = sum w x (x) x, x taken from the w-weighted
 *   barycentre of the boxel's fine voxels (the least-squares plane through the
 *   interface voxels), its sign set by Eq. normal:flip so that N points out of
 *   the inclusion.
 * method COMBO_NORMAL_KABEL: N = Ntilde of Eq. normal:kabel (the direction
 *   from the inclusion's barycentre to the matrix's), the comparison method
 *   of Sec. 5; where the two barycentres coincide, the Laplacian normal.
 * In both, where the barycentres coincide the sign of the Laplacian normal is
 * the eigen-solver's (Eq. normal:flip cannot decide it).
 *
 * The outputs feed combo_problem directly (phase, boxel_idx, boxel_N,
 * boxel_c).
 *   n[3], b[3]  fine grid and boxel sizes in fine voxels (host).
 *   h[3]        fine voxel edges, > 0 (host).
 *   chi         [n3][n2][n1] bytes, x fastest; nonzero = inclusion.  In `mem`.
 *   phase_out   [nc1 nc2 nc3] phase codes, coarse index I + nc1 (J + nc2 K).
 *   idx_out     [cap] coarse indices of the boxels, increasing.
 *   N_out       [cap][3] unit normals; c_out [cap] c+ (FP64).
 *   n_boxels    host: receives the number of boxels; only the first
 *               min(cap, *n_boxels) are written (cap = 0 counts only; the
 *               boxel pointers may then be NULL).
 *   mem         COMBO_MEM_HOST or COMBO_MEM_DEVICE for chi and the outputs.
 * Limits (else COMBO_E_INVALID_ARG): 2 b1 b2 b3 max(b_j)^2 < 2^31 (the
 * moments are exact integer sums) and (b2 + 2)(b3 + 2)(ceil(n1 / 32) + 1)
 * 4 bytes + 8 nc1 bytes <= 200 KiB (one slab of fine rows with its halo in
 * shared memory).
 * Runs on the context's stream and synchronises it before returning.
 */
#define COMBO_NORMAL_LAPLACE 0
#define COMBO_NORMAL_KABEL 1
int combo_coarse_grain(combo_ctx* ctx, const int32_t n[3], const int32_t b[3], const double h[3], int32_t method,
                       const uint8_t* chi, uint8_t* phase_out, int64_t cap, int64_t* idx_out, double* N_out,
                       double* c_out, int64_t* n_boxels, int32_t mem);

/*
 * Event timing of combo_coarse_grain's kernels, for benchmarks (no
 * counterpart in the paper).  While enabled (per process), each call records
 * CUDA events on its stream around its five launches -- the packing of the
 * image to bits, the slab pass (counts, integer moments), the scan of the
 * per-slab counts, the scatter of the boxel indices and the per-boxel finish
 * (normal, c+) -- and combo_coarse_grain_profile_read gives the last call's
 * durations in ms (ms[0..4]).  Returns COMBO_OK, or COMBO_E_INVALID_ARG when
 * nothing was recorded yet.
 */
int combo_coarse_grain_profile(int32_t enable);
int combo_coarse_grain_profile_read(double ms[5]);

/*
 * Fault injection for tests of the failure paths (no counterpart in the
 * paper).  combo_fault_inject_alloc(k), k >= 0: the device allocations of
 * solves, batches and servers set up afterwards succeed k more times, then
 * one fails as cudaMalloc does when the device is out of memory (the hook
 * then disarms); the call that hit it frees what it had allocated and
 * returns COMBO_E_OOM (combo_solve, combo_solve_begin, combo_solve_batch).
 * k < 0 disarms the hook.  Process-wide; returns COMBO_OK.
 */
int combo_fault_inject_alloc(int64_t after);

/*
 * combo_apply_G_noalloc: the Green operator of combo_apply_G (FP64) for the
 * rotated and spectral schemes, for callers that cannot allocate device memory -- code that runs inside a
 * memory arena or pool it does not own, a loop that must not allocate, or a
 * host framework that owns all device memory.  It has no counterpart in the
 * paper; it is a deployment variant of the Green-operator entry point.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The caller
 * passes X and Y, [9][V] FP64 in device memory (they may be the same buffer).  The
 * half spectrum, the reduction partials, the solver scalars and the
 * twiddle / symbol tables live in one library-owned device array of 4 MiB,
 * which every GPU that loads libcombo.so holds until the process exits; each
 * call fills the tables on the device (no host copy).
 * Limits: each side 2^a 3^b in [2, 64], n1 even, kspace COMBO_ROTATED or
 * COMBO_SPECTRAL (not the staggered grid), and
 * 9 n3 n2 (n1/2 + 1 rounded up to 4) <= 259520 (every grid up to 32^3 fits);
 * anything else returns COMBO_E_INVALID_ARG with a message.
 *   device  CUDA device ordinal to run on (made current for the call).
 *   stream  cudaStream_t (NULL = the default stream).
 *   sumsq   optional host pointer: receives sum_x |Y(x)|^2; when given, the
 *           call synchronises the stream before it returns.
 * The first call on a device looks up the array's device address (a
 * synchronous runtime query).  Every call on a device shares the
 * array and finds the previous call's contents there (it clears what must
 * start at zero): calls that overlap on the GPU -- on different streams, or
 * from several threads -- race and must be serialised by the caller.
 */
int combo_apply_G_noalloc(int32_t device, void* stream, const int32_t n[3], const double l[3], int32_t kspace,
                          const double* X, double* Y, double* sumsq);

#ifdef __cplusplus
}
#endif
#endif

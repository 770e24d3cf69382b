/*
 * pimpc.h -- C ABI of the GB300 (sm_103a) piMPC solver library.
 *
 * The library runs the hot path of piMPC (Wu et al., "piMPC: A Parallel-in-horizon and
 * Construction-free NMPC Solver", arXiv 2601.14414): the velocity-form, construction-free ADMM
 * iteration of Algorithm 1 on a batch of independent MPC instances, plus the real-time-iteration
 * pieces around it (explicit-Euler relinearisation, the per-stage factorisations the iteration
 * caches, the plant step) and a reverse-mode adjoint of the unrolled iteration.
 *
 * Problem (Sec. II, problem statement): for each instance
 *   min  sum_k 1/2 ||x_{k+1} - r_x||^2_Q + 1/2 ||u_k - r_u||^2_R  (+ 1/2 ||u_k - u_{k-1}||^2_Wdu)
 *   s.t. x_{k+1} = A_k x_k + B_k u_k + e_k,  xmin <= x_{k+1} <= xmax,  umin <= u_k <= umax,
 *        x_0 = x(t),  k = 0..N-1,
 * with Q, R, Wdu diagonal (C = I). The solver works on the velocity form of Theorem 2,
 * xbar_k = (x_k, u_{k-1}), n = nx + nu.
 *
 * Conventions for every call:
 *   - Plain C types only. Every array argument is FP64, row-major, instances concatenated in
 *     batch order, each instance's part stage-major. `mem` says whether the pointers are host
 *     (PIMPC_HOST) or device (PIMPC_DEVICE) memory of the solver's device. `stream` is a
 *     cudaStream_t (NULL = legacy default stream); device-memory calls are asynchronous on it;
 *     host-memory calls copy with cudaMemcpyAsync on it and synchronise it before returning.
 *   - Ownership: the caller owns every buffer it passes and may free or reuse it when the call
 *     returns (host memory) or when the stream has passed the call (device memory). The solver
 *     owns all device state (matrices, caches, iterates); pimpc_create allocates all of it
 *     except the adjoint's checkpoint store, which the first pimpc_backward call allocates, the
 *     input-set arrays (first pimpc_set_input_set call) and the buffer of the testing aid
 *     pimpc_set_restart_mask; pimpc_destroy frees everything.
 *   - Errors: a nonzero return means the call did nothing (arguments are validated before any
 *     launch) except PIMPC_ECUDA, which reports a CUDA error; pimpc_last_error(s) then holds a
 *     message. Non-convergence is not an error: it is reported per instance in `status`.
 *   - One solver object serves one stream at a time; calls on one object are not thread-safe.
 */
#ifndef PIMPC_H
#define PIMPC_H

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum { PIMPC_OK = 0, PIMPC_EINVAL = 1, PIMPC_ENOMEM = 2, PIMPC_ECUDA = 3, PIMPC_ESTATE = 4 };
/* Per-instance solve status. */
enum {
  PIMPC_CONVERGED = 0,      /* c^{i+1} <= eps (Algorithm 1 step 5)                          */
  PIMPC_MAXITER = 1,        /* max_iters reached                                            */
  PIMPC_NONFINITE = 2,      /* c^{i+1} is not finite                                        */
  PIMPC_TIMEOUT = 3,        /* a bounded wait of the launch gave up before the instance ended */
  PIMPC_FACTOR_FAILED = 4,  /* the stage cache met a non-positive (or NaN) pivot: non-finite  */
                            /* or overflowing dynamics; the instance's outputs are not valid  */
  PIMPC_STALLED = 5         /* c stopped decreasing (pimpc_set_stall): the arithmetic's floor */
};
/* Arithmetic of the ADMM iterations (the factorisation is always FP64). */
enum { PIMPC_F32 = 0, PIMPC_F64 = 1 };
/* Memory space of caller buffers. */
enum { PIMPC_HOST = 0, PIMPC_DEVICE = 1 };
/* Built-in nonlinear models for pimpc_linearise / pimpc_plant_step. */
enum { PIMPC_MODEL_QUADROTOR = 0, PIMPC_MODEL_CARTPOLE = 1, PIMPC_MODEL_CSTR = 2 };

/* Size limits of one instance. */
#define PIMPC_MAX_N_LTV 32   /* n = nx + nu for stage-varying dynamics   */
#define PIMPC_MAX_N_LTI 64   /* n = nx + nu for stage-invariant dynamics */
#define PIMPC_MAX_NU 32      /* nu (inputs per stage), any dynamics      */

typedef struct pimpc_solver pimpc_solver;

/*
 * pimpc_create -- setup(model dims, N): allocate a solver for `batch` independent instances.
 *   nx[batch], nu[batch], N[batch]  host arrays: state size (>= 1), input size (>= 1) and horizon
 *                                   (>= 1) of each instance; n = nx + nu <= PIMPC_MAX_N_LTV
 *                                   (lti = 0) or PIMPC_MAX_N_LTI (lti = 1), nu <= PIMPC_MAX_NU.
 *   lti        1: one (A, B, e) per instance used at every stage; 0: one triple per stage.
 *   precision  PIMPC_F32 or PIMPC_F64 arithmetic for the iterations.
 *   device     CUDA device ordinal.
 *   out        receives the solver (NULL on failure).
 * Defaults after create: rho = 1, eps = 1e-6, max_iters = 1000, accel = 1, eta = 0.999
 * (Algorithm 1), zero weights, infinite bounds, zero dynamics, cold start.
 * Errors: PIMPC_EINVAL (sizes), PIMPC_ENOMEM, PIMPC_ECUDA. On failure the message is returned
 * by pimpc_last_error(NULL) on the calling thread.
 */
int pimpc_create(int batch, const int *nx, const int *nu, const int *N, int lti, int precision,
                 int device, pimpc_solver **out);

/* Free all device and host memory of the solver; synchronises its last stream. NULL is a no-op. */
void pimpc_destroy(pimpc_solver *s);

/* Message of the last failed call on `s` ("" if none); with s == NULL, of the last failed
 * pimpc_create on this thread. The string lives until the next call on the same object. */
const char *pimpc_last_error(const pimpc_solver *s);

/*
 * pimpc_set_weights -- setup(Q, R): cost weights Qbar = diag(q, r) of Theorem 2.
 *   q[sum nx]    diagonal of C^T W_y C (>= 0);  r[sum nu] diagonal of W_u (>= 0);
 *   rdu[sum nu]  diagonal of an optional weight on u_k - u_{k-1} (>= 0), NULL = 0 (Algorithm 1).
 * Marks the factorisation stale. Errors: PIMPC_EINVAL for a negative or non-finite entry.
 */
int pimpc_set_weights(pimpc_solver *s, const double *q, const double *r, const double *rdu,
                      int mem, void *stream);

/*
 * pimpc_set_bounds -- setup(bounds): the box Xbar = X x U of Theorem 2, same for every stage.
 *   xmin, xmax [sum nx]; umin, umax [sum nu]; +-INFINITY allowed, NaN not.
 * Errors: PIMPC_EINVAL if some lower bound exceeds its upper bound.
 */
int pimpc_set_bounds(pimpc_solver *s, const double *xmin, const double *xmax, const double *umin,
                     const double *umax, int mem, void *stream);

/*
 * pimpc_set_options -- setup(rho) and the iteration controls of Algorithm 1.
 *   rho > 0 (penalty; a change marks the factorisation stale), eps (stop when c^{i+1} <= eps,
 *   step 5; eps < 0 never stops early), max_iters >= 0 (K_max), accel (0: plain iteration,
 *   1: accelerated with restart, steps 6-7), eta (restart threshold, 0.999 in Algorithm 1).
 * Errors: PIMPC_EINVAL.
 */
int pimpc_set_options(pimpc_solver *s, double rho, double eps, int max_iters, int accel,
                      double eta);

/*
 * pimpc_set_dynamics -- construction-free input: the stage matrices themselves (Sec. II).
 *   A [sum N nx nx] (lti: [sum nx nx]), B [sum N nx nu] (lti: [sum nx nu]),
 *   e [sum N nx] (lti: [sum nx]); e may be NULL (= 0).
 * Marks the factorisation stale. Errors: PIMPC_EINVAL.
 */
int pimpc_set_dynamics(pimpc_solver *s, const double *A, const double *B, const double *e,
                       int mem, void *stream);

/*
 * pimpc_linearise -- linearise(xbar, ubar): explicit-Euler linearisation of a built-in model
 * along a trajectory (the real-time-iteration scheme the paper's NMPC uses, Sec. I and Sec. V-C):
 *   A_k = I + dt df/dx, B_k = dt df/du, e_k = F(xbar_k, ubar_k) - A_k xbar_k - B_k ubar_k,
 *   F(x, u) = x + dt f(x, u), evaluated at (xbar_k, ubar_k), k = 0..N-1.
 *   model   PIMPC_MODEL_*; every instance must have that model's (nx, nu).
 *   params  [batch][P] model parameters (quadrotor P = 7: m, g, Jx, Jy, Jz, l, k_yaw;
 *           cart-pole P = 4: m_cart, m_pole, half-length, g; CSTR P = 4: C_Ai, k0, EaR, T_i).
 *   xbar [sum N nx], ubar [sum N nu]  linearisation points (lti = 1: [sum nx], [sum nu]).
 *   dt > 0.
 * Replaces the dynamics and marks the factorisation stale. Errors: PIMPC_EINVAL.
 */
int pimpc_linearise(pimpc_solver *s, int model, const double *params, double dt,
                    const double *xbar, const double *ubar, int mem, void *stream);

/*
 * pimpc_get_dynamics -- copy out the stage matrices in use (as set by pimpc_set_dynamics or
 * produced by pimpc_linearise), FP64, in the layout of pimpc_set_dynamics. Any pointer may be NULL.
 */
int pimpc_get_dynamics(pimpc_solver *s, double *A, double *B, double *e, int mem, void *stream);

/*
 * pimpc_factorise -- the per-stage cache of Algorithm 1 in FP64: for every stage,
 *   H_k = (Qbar + rho I + rho Abar_{k+1}^T Abar_{k+1})^{-1} (k < N-1), H_{N-1} = (Qbar + rho I)^{-1}
 *   (definition after the velocity-form iteration) and M_k = (B_k^T B_k + I + Wdu / rho)^{-1},
 *   so that J_k v = M_k Bbar_k^T v, inverted by Gauss-Jordan sweeps of the symmetric matrix in
 *   pivot order (no pivoting: both matrices are positive definite). Results are stored in the
 *   iteration precision. pimpc_solve calls it implicitly when the cache is stale. With valid
 *   weights and rho both matrices are >= I (symmetric positive definite), so a non-positive
 *   pivot means non-finite or overflowing dynamics: the call stays asynchronous and the next
 *   solve reports such instances with status PIMPC_FACTOR_FAILED.
 * Errors: PIMPC_ECUDA.
 */
int pimpc_factorise(pimpc_solver *s, void *stream);

/*
 * pimpc_solve -- solve(x0, ref, iters | tol): Algorithm 1 on every instance.
 *   x0 [sum nx]          measured state x(t).
 *   u_prev [sum nu]      u(t-1) in xbar_0 = (x(t), u(t-1)); NULL = 0 (Algorithm 1 input).
 *   ref                  reference of xbar_{k+1} = (x_{k+1}, u_k): [sum N n] if ref_per_stage,
 *                        else [sum n]; qbar_k = Qbar ref_k. NULL = 0.
 *   warm_start           0: cold start (all iterates 0); 1: start from the iterates the previous
 *                        solve left (Algorithm 1 output); 2: the same, shifted one stage earlier
 *                        with the last stage repeated.
 *   u_out [sum N nu], x_out [sum N nx]   u_k and x_{k+1} read from z_{k+1} (inside the box);
 *                        either may be NULL.
 *   iters[batch], c[batch], status[batch]  iterations run, last c^{i+1}, PIMPC_CONVERGED /
 *                        MAXITER / NONFINITE / TIMEOUT / FACTOR_FAILED / STALLED; any may
 *                        be NULL.
 * Errors: PIMPC_EINVAL, PIMPC_ECUDA.
 */
int pimpc_solve(pimpc_solver *s, const double *x0, const double *u_prev, const double *ref,
                int ref_per_stage, int warm_start, double *u_out, double *x_out, int *iters,
                double *c, int *status, int mem, void *stream);

/*
 * pimpc_set_graph -- CUDA graphs for device-memory solves (enable = 1) or direct launches
 * (enable = 0, the default). With graphs on, the launches of a pimpc_solve with mem ==
 * PIMPC_DEVICE are recorded into a CUDA graph the first time an argument set (the pointers,
 * ref_per_stage, warm_start, polish on or off) is seen and replayed by later calls with the same
 * set: one graph launch per solve. The stage cache, when stale, is rebuilt outside the graph
 * before the launch. A call that changes launch parameters (set_options, set_schedule,
 * set_polish, set_restart_mask) drops the recorded graphs. If the driver refuses the capture,
 * that call and later ones run the launches directly (pimpc_get_graph_stats reports why).
 * Host-memory solves always launch directly. Errors: PIMPC_EINVAL.
 */
int pimpc_set_graph(pimpc_solver *s, int enable);

/*
 * pimpc_get_graph_stats -- whether graphs are in use, how many graphs were captured and how
 * many solves replayed one, and (when the capture was refused) the driver's reason (owned by the
 * solver, valid until the next call on it; NULL otherwise). Any pointer may be NULL.
 */
int pimpc_get_graph_stats(pimpc_solver *s, int *enabled, long long *captures, long long *replays,
                          const char **refused);

/*
 * pimpc_set_polish -- FP64 polish of FP32 solves: after the FP32 iterations stop (eps or
 * max_iters), up to polish_iters further iterations run in FP64 (FP64 stage cache, FP64 residual
 * c) from the FP32 iterates, stopping on c <= polish_eps; u_out and x_out are then the polished
 * FP64 results and the per-instance iters, c and status of pimpc_solve / pimpc_get_stats are
 * (FP32 iterations + polish iterations, the polish's c, the polish's status). polish_iters = 0
 * (the default) turns it off; solvers with FP64 iterations ignore it. The first polished solve
 * creates an FP64 copy of the stage cache and iterate buffers (about twice the FP32 memory).
 * pimpc_get_iterates keeps returning the FP32 iterates, and warm starts reuse them.
 * Errors: PIMPC_EINVAL (polish_iters < 0, NaN polish_eps).
 */
int pimpc_set_polish(pimpc_solver *s, int polish_iters, double polish_eps);

/*
 * pimpc_get_iterates -- copy the iterates the last solve ended with (the non-hat iterates that
 * Algorithm 1 outputs for warm start): z, v, theta, beta, lambda, each [sum N n], with
 * z[k] = z_{k+1}, v[k] = v_k, theta[k] = theta_k, ... Any pointer may be NULL.
 * Errors: PIMPC_ESTATE before the first solve.
 */
int pimpc_get_iterates(pimpc_solver *s, double *z, double *v, double *theta, double *beta,
                       double *lambda, int mem, void *stream);

/*
 * pimpc_get_stats -- per-instance results of the last solve: iters[batch], c[batch] (last
 * c^{i+1}), status[batch], momentum_iters[batch] (iterations whose hats used the momentum step
 * of Algorithm 1 step 6, i.e. read the iterate before the current one). Any pointer may be NULL.
 * Errors: PIMPC_ESTATE before the first solve.
 */
int pimpc_get_stats(pimpc_solver *s, int *iters, double *c, int *status, int *momentum_iters,
                    int mem, void *stream);

/*
 * pimpc_set_restart_mask -- replay fixed restart decisions (testing aid): mask[batch][len],
 * 1 = momentum step, 0 = restart, used for iteration i < len instead of c^{i+1} <= eta c^i;
 * NULL clears it. Errors: PIMPC_EINVAL (len < 0 or len > max_iters).
 */
int pimpc_set_restart_mask(pimpc_solver *s, const unsigned char *mask, int len, int mem,
                           void *stream);

/*
 * pimpc_set_input_set -- the input part of Xbar = X x U as a non-box convex set (the remark after
 * Theorem 1: the (v, z) update of the splitting stays a Euclidean projection for any closed
 * convex set, so only the projection of z's input part changes). Per instance:
 *   kind[batch]  0: the box [umin, umax] (pimpc_set_bounds; the default), 1: l2 ball
 *                ||u||_2 <= r, 2: l1 ball ||u||_1 <= r, 3: halfspace a^T u <= r, 4: second-order
 *                cone ||(u_1, .., u_{nu-1})||_2 <= u_0. For kinds 1-4 the input box is not used;
 *                the state box always is.
 *   r[batch]     radius (kinds 1, 2: finite, >= 0) or offset (kind 3: finite); unused otherwise.
 *   a[sum nu]    halfspace normals (kind 3: finite, nonzero); may be NULL if no instance has
 *                kind 3.
 * Sets hold for every stage of the instance. Schedules: families 0 and 5 (the defaults) only;
 * pimpc_set_schedule and pimpc_autotune keep to them while a non-box set is in force, and
 * pimpc_backward (box only) returns PIMPC_ESTATE. The first call allocates the set arrays. The
 * call synchronises `stream`.
 * Errors: PIMPC_EINVAL (a bad kind or parameter, or a schedule family other than 0 or 5 in
 * force), PIMPC_ENOMEM, PIMPC_ECUDA.
 */
int pimpc_set_input_set(pimpc_solver *s, const int *kind, const double *r, const double *a,
                        int mem, void *stream);

/*
 * pimpc_set_stall -- a second stop test beside Algorithm 1's c <= eps (no counterpart in the
 * paper; for FP32 iterations): once an instance's c^{i+1} has come below `below` (first at
 * iteration i0), it also stops, with status PIMPC_STALLED, when c has not fallen below factor x
 * the smallest c seen since for max(window, rel x i0) consecutive iterations (an instance that
 * needed many iterations to get there converges slowly and keeps improving its iterates for
 * longer after its c has levelled off). In FP32 the residual c of a slowly converging instance levels
 * off where the rounding of the iterates outweighs their change (about 1e-11 to 1e-10 on the
 * batched workloads) while its iterates are already as accurate as FP32 makes them; a tolerance
 * eps set below that floor then ends such instances here instead of at max_iters. `below` keeps
 * the plateaus of the accelerated iteration far above the floor from counting. window = 0 (the
 * default) turns the test off. Errors: PIMPC_EINVAL (window < 0, factor outside (0, 1],
 * below < 0 or NaN, rel < 0 or not finite).
 */
int pimpc_set_stall(pimpc_solver *s, int window, double factor, double below, double rel);

/*
 * pimpc_set_wait_limit -- bound of the grid-wide barrier of the persistent launch (testing aid,
 * no counterpart in the paper): a CTA polls the barrier at most `polls` times (about 0.1 us
 * each) before the launch gives up, stops every CTA at its next barrier and reports the
 * instances it did not finish as PIMPC_TIMEOUT. 0 (the default) restores the built-in limit
 * (about half a second). Affects the schedule families with a grid barrier (0, 2, 4, 5).
 * Errors: PIMPC_EINVAL (polls < 0).
 */
int pimpc_set_wait_limit(pimpc_solver *s, int polls);

/*
 * pimpc_plant_step -- one explicit-Euler step x_next = x + dt f(x, u) of a built-in model per
 * instance (the closed-loop plant of the real-time-iteration loop).
 *   params [batch][P], x [sum nx], u [sum nu], x_next [sum nx].
 * Errors: PIMPC_EINVAL.
 */
int pimpc_plant_step(pimpc_solver *s, int model, const double *params, double dt,
                     const double *x, const double *u, double *x_next, int mem, void *stream);

/*
 * pimpc_backward -- reverse mode of the unrolled iteration (an extension the paper names as
 * future work, Sec. VI): given the loss gradients w.r.t. the outputs of the last pimpc_solve,
 * returns the gradients w.r.t. its inputs. The last solve must have used warm_start = 0,
 * accel = 0 and eps < 0 (a fixed number of iterations, so that the map is the unrolled one).
 *   dL_du [sum N nu], dL_dx [sum N nx]   gradients w.r.t. u_out, x_out.
 *   g_x0 [sum nx], g_ref [sum N n] (per-stage reference) or [sum n] (constant reference,
 *   following the ref_per_stage of the last solve), g_q [sum nx], g_r [sum nu],
 *   g_xmin, g_xmax [sum nx], g_umin, g_umax [sum nu]; any may be NULL.
 *   checkpoint_every  forward states kept every K iterations (K >= 1); the other iterations
 *                     are recomputed segment by segment.
 * Errors: PIMPC_ESTATE (no suitable solve), PIMPC_EINVAL, PIMPC_ENOMEM (checkpoint store),
 * PIMPC_ECUDA.
 */
int pimpc_backward(pimpc_solver *s, const double *dL_du, const double *dL_dx, double *g_x0,
                   double *g_ref, double *g_q, double *g_r, double *g_xmin, double *g_xmax,
                   double *g_umin, double *g_umax, int checkpoint_every, int mem, void *stream);

/*
 * Schedules of the batched solve (no counterpart in the paper: how the GPU cuts the work of
 * Algorithm 1 across its SMs; the arithmetic of an iteration is the same under every schedule,
 * up to the order of the sums in c).
 *   family       0: a group of lanes per stage on plain stage blocks, one component per lane
 *                   (every precision and instance kind; the default for FP64 iterations);
 *                   2: one thread per stage on halo tiles (stage-varying FP32 instances only);
 *                   3: every instance resident in the shared memory of one CTA or of a
 *                   thread-block cluster for the whole solve (no grid-wide synchronisation;
 *                   for instances that fit); 4: stage-invariant instances only, the per-stage
 *                   products of blocks of stages as dense matrix-matrix contractions; 5: a
 *                   group of 4, 8 or 16 lanes per stage on blocked stage blocks, four
 *                   components per lane (every precision and instance kind; the default for
 *                   FP32 iterations); 6: stage-invariant instances with FP32 iterations, the
 *                   per-stage products of 127-stage tiles as matrix products on the tensor
 *                   cores (tcgen05, TF32 operands split in two for FP32 accuracy; nx and nu
 *                   rounded up to 16 must sum to 64 or less, nu's at most nx's); 7: temporal
 *                   blocking of the plain iteration (accel = 0 only): windows of stages loaded
 *                   once into shared memory, iterated T times there with T halo stages on each
 *                   open side and written back on their interior, the stop test every T
 *                   iterations; -1: the default.
 *   ctas_per_sm  families 2, 4, 5 and 7: CTAs per SM the shared-memory budget of a CTA is sized
 *                for (0 = 2 for family 2, 1 for family 4; for family 5 the one of 3, 2, 1 that
 *                fits every instance with the most stages in flight); ignored by families 0
 *                and 3.
 *   item_scale   families 0 and 5: stage sub-chunks per work item (0 = automatic; when the
 *                active items no longer cover the grid the solve switches to items of one
 *                sub-chunk for stage-varying batches); family 2: at most
 *                this many tiles per work item (0 = 4); family 3: CTAs per instance, 1, 2, 4,
 *                8 or 16 (0 = the fewest whose shared memory holds the instance, or the most
 *                that leave each CTA four stages when the batch occupies few SMs); family 4:
 *                stages per block (0 = as many as the shared memory holds, at most 128);
 *                family 6: 127-stage tiles per work item (0 = 2); family 7: T, iterations per
 *                block (0 = 8).
 * pimpc_set_schedule re-lays out the stage data and the iterates: the next solve factorises
 * again and starts cold (warm_start is treated as 0 until one solve has run).
 * Errors: PIMPC_EINVAL (a bad value, or an instance that does not fit the schedule; the
 * previous schedule stays in force), PIMPC_ENOMEM, PIMPC_ECUDA.
 */
int pimpc_set_schedule(pimpc_solver *s, int family, int ctas_per_sm, int item_scale);

/*
 * pimpc_get_schedule -- the schedule in force and the launch it gives: grid (CTAs of the
 * persistent launch), threads (per CTA) and items (work items of one iteration over the whole
 * batch). Any pointer may be NULL (host memory).
 */
int pimpc_get_schedule(pimpc_solver *s, int *family, int *ctas_per_sm, int *item_scale,
                       int *grid, int *threads, int *items);

/*
 * pimpc_autotune -- times trial_iters iterations (zero start, no reference, the accel option in
 * force) of every candidate schedule on this solver's batch, with its current dynamics, weights
 * and bounds, using CUDA events on `stream`, and keeps the fastest. Candidates: family 0 with
 * item_scale 0, 2 and 8; family 5 with 2, 3 and 4 CTAs per SM; family 3 where the instances
 * fit; family 4 for stage-invariant batches; family 2 with 1 and 2 CTAs per SM where the batch
 * allows it. The
 * chosen schedule and its time (ms, the second of two trial solves) are returned through the
 * pointers (host memory, any may be NULL). The stage cache and the iterates are rebuilt as for
 * pimpc_set_schedule. Blocks the host until the trials finish.
 * Errors: PIMPC_EINVAL (trial_iters < 1), PIMPC_ENOMEM, PIMPC_ECUDA.
 */
int pimpc_autotune(pimpc_solver *s, int trial_iters, int *family, int *ctas_per_sm,
                   int *item_scale, double *best_ms, void *stream);

/*
 * pimpc_solve_static -- one instance, solved without allocating any device memory.
 *
 * No counterpart in the paper: this entry point exists for callers that cannot call cudaMalloc
 * (real-time control loops that forbid allocation after start-up, because an allocation can
 * synchronise the device and has no latency bound; controllers certified without dynamic
 * memory; plug-ins inside a host whose device memory belongs to another framework). It
 * computes what pimpc_create + set_* + pimpc_solve (cold start) compute for a single
 * stage-varying instance, with the same kernels, but its working memory is one file-scope
 * device array of PIMPC_STATIC_BYTES that every GPU loading the library holds until exit.
 *   nx, nu, N     sizes, 1 <= nx, 1 <= nu, nx + nu <= PIMPC_MAX_N_LTV, N >= 1.
 *   precision     PIMPC_F32 or PIMPC_F64 iterations (factorisation in FP64).
 *   A [N nx nx], B [N nx nu], e [N nx] (NULL = 0), q [nx], r [nu], xmin, xmax [nx],
 *   umin, umax [nu], x0 [nx], ref [n] (constant reference, NULL = 0): DEVICE memory, FP64,
 *   owned by the caller, read during the call's kernels only.
 *   rho, eps, max_iters, accel, eta  as in pimpc_set_options, with the same checks.
 *   u_out [N nu], x_out [N nx], iters[1], c[1], status[1]: DEVICE memory (any may be NULL).
 *   stream        cudaStream_t; the call only enqueues work on it.
 * The call allocates nothing (no cudaMalloc, no cudaFree, no allocating library call). Its
 * first call on a device looks up the array's address with cudaGetSymbolAddress; make that
 * first call before any stream capture. Every call shares the array and rewrites or clears what
 * it reads, so consecutive calls are independent, but calls that overlap on the GPU race.
 * Capacity: the working memory is about N * (W + 15 n) * ts bytes (ts = 4 in FP32, 8 in FP64;
 * W = nx n + nx + n(n+1)/2 + nu(nu+1)/2 words of stage data, N rounded up to a multiple of 32),
 * so at n = 32 the worst split (nx = 31, nu = 1, W = 1552) fits about 2000 stages in FP32 and
 * 1000 in FP64.
 * Errors: PIMPC_EINVAL (sizes, options, or an instance whose working memory exceeds
 * PIMPC_STATIC_BYTES; the message is in pimpc_last_error(NULL)), PIMPC_ECUDA.
 */
#define PIMPC_STATIC_BYTES (16u << 20)
int pimpc_solve_static(int nx, int nu, int N, int precision, const double *A, const double *B,
                       const double *e, const double *q, const double *r, const double *xmin,
                       const double *xmax, const double *umin, const double *umax,
                       const double *x0, const double *ref, double rho, double eps,
                       int max_iters, int accel, double eta, double *u_out, double *x_out,
                       int *iters, double *c, int *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PIMPC_H */

/*
 * pimpc_oracle.h -- plain FP64 CPU oracle for the piMPC hot path (arXiv 2601.14414).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference leg may load the library built from this header. The product library neither
 * includes this header nor links the oracle; the two share no code, header, table or constant.
 *
 * Conventions (all arrays row-major, FP64, one MPC instance per call):
 *   nx, nu     state and input sizes; n = nx + nu is the velocity-form state size (Theorem 2).
 *   N          horizon length; "stage k" means k = 0..N-1.
 *   A[N][nx][nx], B[N][nx][nu], e[N][nx]   stage matrices of x_{k+1} = A_k x_k + B_k u_k + e_k
 *                                          (problem statement, Sec. II).
 *   q[nx], r[nu]    diagonals of C^T W_y C and W_u, so Qbar = diag(q, r) (Theorem 2).
 *   rdu[nu]         diagonal of an optional W_du weight on du (NULL = 0; Algorithm 1 has none).
 *   ref[N][n]       reference for xbar_{k+1} = (x_{k+1}, u_k); qbar_k = Qbar * ref[k].
 *   bounds          the box Xbar = X x U of Theorem 2: lo = (xmin, umin), hi = (xmax, umax);
 *                   +-INFINITY allowed.
 *   uset            the input set U (the remark after Theorem 1: the (v, z) update stays a
 *                   Euclidean projection for any closed convex set): ORC_USET_BOX (the box
 *                   [umin, umax], the default), ORC_USET_BALL2 (||u||_2 <= uset_r),
 *                   ORC_USET_BALL1 (||u||_1 <= uset_r), ORC_USET_HALFSPACE (uset_a^T u <=
 *                   uset_r, uset_a[nu] nonzero), ORC_USET_SOC (||u_{1:nu-1}||_2 <= u_0, the
 *                   second-order cone); umin and umax are ignored for the non-box sets.
 *   iterates        array index k holds: z[k] = z_{k+1}, v[k] = v_k, th[k] = theta_k,
 *                   be[k] = beta_k, la[k] = lambda_k (all [N][n]), du[k] = du_k ([N][nu]),
 *                   xb[k] = xbar_{k+1} ([N][n]).
 */
#ifndef PIMPC_ORACLE_H
#define PIMPC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, nu, N;
  const double *A, *B, *e;
  const double *q, *r, *rdu;
  const double *xmin, *xmax, *umin, *umax;
  const double *x0, *u_prev;
  const double *ref;
  double rho;
  int uset;
  double uset_r;
  const double *uset_a;
} orc_problem;

enum { ORC_USET_BOX = 0, ORC_USET_BALL2 = 1, ORC_USET_BALL1 = 2, ORC_USET_HALFSPACE = 3,
       ORC_USET_SOC = 4 };

typedef struct {
  double eps;                      /* stop when c^{i+1} <= eps (Algorithm 1, step 5)       */
  int max_iters;                   /* K_max                                                */
  int accel;                       /* 0: plain iteration (hats = iterates); 1: steps 6-7    */
  double eta;                      /* restart threshold, 0.999 in Algorithm 1              */
  const unsigned char *force_mask; /* NULL, or [max_iters]: 1 = momentum, 0 = restart      */
} orc_options;

enum { ORC_CONVERGED = 0, ORC_MAXITER = 1, ORC_NONFINITE = 2 };

/* Euclidean projection of y[nu] onto the input set of p (out[nu]). Returns 0 or -1. */
int orc_project_u(const orc_problem *p, const double *y, double *out);

/* Explicit per-stage cache of Algorithm 1: H[N][n][n] and J[N][nu][n]. Returns 0 or -1. */
int orc_cache(const orc_problem *p, double *H, double *J);

/* One pass of Algorithm 1 steps 1-4 from the hats (zh, vh, thh, beh, lah). Writes du, xb and
 * the new iterates; returns c^{i+1} through *c. Returns 0 or -1. */
int orc_iteration(const orc_problem *p, const double *H, const double *J,
                  const double *zh, const double *vh, const double *thh, const double *beh,
                  const double *lah, double *du, double *xb, double *z, double *v, double *th,
                  double *be, double *la, double *c);

/* Algorithm 1. z, v, th, be, la hold the starting iterates on entry (all zero = cold start) and
 * the final non-hat iterates on exit. c_hist and mask_hist may be NULL, else [max_iters]. */
int orc_solve(const orc_problem *p, const orc_options *o, double *z, double *v, double *th,
              double *be, double *la, double *du, double *xb, int *iters, double *c_final,
              int *status, double *c_hist, unsigned char *mask_hist);

/* Built-in nonlinear models for the real-time-iteration loop. */
enum { ORC_MODEL_QUADROTOR = 0, ORC_MODEL_CARTPOLE = 1, ORC_MODEL_CSTR = 2 };
int orc_model_dims(int model, int *nx, int *nu);
/* Continuous-time right-hand side f(x, u). */
int orc_model_f(int model, const double *params, const double *x, const double *u, double *f);
/* Explicit-Euler linearisation along (xbar[N][nx], ubar[N][nu]):
 * A_k = I + dt df/dx, B_k = dt df/du, e_k = F(xbar_k, ubar_k) - A_k xbar_k - B_k ubar_k with
 * F(x, u) = x + dt f(x, u). Jacobians by the complex-step derivative. */
int orc_linearise(int model, const double *params, double dt, int N, const double *xbar,
                  const double *ubar, double *A, double *B, double *e);
/* One explicit-Euler plant step x_next = x + dt f(x, u). */
int orc_plant_step(int model, const double *params, double dt, const double *x, const double *u,
                   double *x_next);

#ifdef __cplusplus
}
#endif
#endif

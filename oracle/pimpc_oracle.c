/*
 * pimpc_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the piMPC hot path
 * (Wu et al., "piMPC: A Parallel-in-horizon and Construction-free NMPC Solver", arXiv 2601.14414).
 *
 * TEST INFRASTRUCTURE ONLY: it exists to check the CUDA path. Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may load it. It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (IEEE FP64, no fused multiply-add, every sum in
 * index order).
 *
 * Nothing here exploits structure. The velocity-form matrices are materialised densely, H_k and
 * J_k are formed as explicit inverses, and every product is a plain loop, so each line can be
 * read against the paper:
 *   Theorem 2:  xbar_k = col(x_k, u_{k-1}), Abar_k = [[A_k, B_k], [0, I]], Bbar_k = [B_k; I],
 *               ebar_k = col(e_k, 0), Qbar = diag(C^T W_y C, W_u), qbar = Qbar * reference.
 *   cache:      J_k = (Bbar_k^T Bbar_k)^{-1} Bbar_k^T (Algorithm 1, "cache"),
 *               H_k = (Qbar + rho I + rho Abar_{k+1}^T Abar_{k+1})^{-1} for k < N-1 and
 *               H_{N-1} = (Qbar + rho I)^{-1} (definition of H_k after the velocity-form iteration).
 *   iteration:  Algorithm 1 steps 1-7.
 *
 * Readings taken where the paper is ambiguous (each is pinned by a test in tests/):
 *   R1  z-update: the argument keeps the Abar_k xbar_k + ebar_k - lambda_k term, i.e. the form the
 *       proof of Theorem 1 derives and Algorithm 1 step 2 prints; the theorem statement drops it.
 *   R2  h_k uses Abar_{k+1} AND ebar_{k+1}: xbar_{k+1} enters the dynamics constraint of stage k+1
 *       (the augmented Lagrangian of the splitting). The printed h_k mixes k and k+1.
 *   R3  the lambda update uses v_k (velocity-form iteration, Algorithm 1 step 3).
 *   R4  in c the hats are those of the same stage: z_{k+1} - zhat_{k+1}, theta_k - thetahat_k, ...
 *   R5  c = rho * (sum of the six SQUARED norms); the stop test is c <= eps.
 *   R6  xbar_0 = col(x(t), u_prev) with u_prev a parameter (default 0, as in Algorithm 1).
 *   R7  restart (Algorithm 1 step 7): hats := current iterates, alpha := 1; the computed c^{i+1} is
 *       kept as the next comparison value; (alpha_i - 1)/alpha_{i+1} uses the pre-update alpha_i.
 *   R8  optional W_du: du_k = (W_du/rho + Bbar^T Bbar)^{-1} Bbar^T (vhat - betahat); W_du = 0 gives
 *       Algorithm 1 exactly.
 *   R9  projection onto the box is min(max(y, lo), hi).
 *   R10 no separate terminal weight: stage N-1 uses the same Qbar.
 *   R11 non-box input sets (the remark after Theorem 1): the reduced (v, z) problem has the
 *       Hessian (3/2) I whatever the set, so z_{k+1} is the Euclidean projection of the same
 *       point; the state part keeps its box, the input part is projected onto U as a vector.
 */
#include "pimpc_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Dense helpers (row-major).                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* y = M x, M is m x n. */
static void mat_vec(int m, int n, const double *M, const double *x, double *y) {
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += M[i * n + j] * x[j];
    y[i] = s;
  }
}

/* y = M^T x, M is m x n. */
static void mat_tvec(int m, int n, const double *M, const double *x, double *y) {
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += M[i * n + j] * x[i];
    y[j] = s;
  }
}

/* C = A^T B, A is m x p, B is m x q, C is p x q. */
static void mat_tmat(int m, int p, int q, const double *A, const double *B, double *C) {
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += A[k * p + i] * B[k * q + j];
      C[i * q + j] = s;
    }
}

/* Minv = M^{-1} by Gauss-Jordan elimination with partial pivoting. Returns -1 if singular. */
static int mat_inverse(int n, const double *M, double *Minv) {
  double *W = (double *)malloc(sizeof(double) * (size_t)n * 2 * n);
  if (!W) return -1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      W[i * 2 * n + j] = (j < n) ? M[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (fabs(W[i * 2 * n + col]) > fabs(W[piv * 2 * n + col])) piv = i;
    if (W[piv * 2 * n + col] == 0.0) { free(W); return -1; }
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        double t = W[col * 2 * n + j];
        W[col * 2 * n + j] = W[piv * 2 * n + j];
        W[piv * 2 * n + j] = t;
      }
    double d = W[col * 2 * n + col];
    for (int j = 0; j < 2 * n; ++j) W[col * 2 * n + j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == col) continue;
      double f = W[i * 2 * n + col];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) W[i * 2 * n + j] -= f * W[col * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Minv[i * n + j] = W[i * 2 * n + n + j];
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Velocity form (Theorem 2).                                                                  */
/* ------------------------------------------------------------------------------------------ */

/* Abar = [[A, B], [0, I]] (n x n), Bbar = [B; I] (n x nu), ebar = col(e, 0) (n). */
static void velocity_form(int nx, int nu, const double *A, const double *B, const double *e,
                          double *Abar, double *Bbar, double *ebar) {
  int n = nx + nu;
  memset(Abar, 0, sizeof(double) * (size_t)n * n);
  memset(Bbar, 0, sizeof(double) * (size_t)n * nu);
  for (int i = 0; i < nx; ++i) {
    for (int j = 0; j < nx; ++j) Abar[i * n + j] = A[i * nx + j];
    for (int j = 0; j < nu; ++j) Abar[i * n + nx + j] = B[i * nu + j];
    for (int j = 0; j < nu; ++j) Bbar[i * nu + j] = B[i * nu + j];
    ebar[i] = e[i];
  }
  for (int j = 0; j < nu; ++j) {
    Abar[(nx + j) * n + nx + j] = 1.0;
    Bbar[(nx + j) * nu + j] = 1.0;
    ebar[nx + j] = 0.0;
  }
}

/* Stage-k views into the problem arrays. */
static const double *stage_A(const orc_problem *p, int k) { return p->A + (size_t)k * p->nx * p->nx; }
static const double *stage_B(const orc_problem *p, int k) { return p->B + (size_t)k * p->nx * p->nu; }
static const double *stage_e(const orc_problem *p, int k) { return p->e + (size_t)k * p->nx; }

/* Qbar = diag(q, r) as a vector of length n. */
static void qbar_diag(const orc_problem *p, double *Qd) {
  for (int i = 0; i < p->nx; ++i) Qd[i] = p->q[i];
  for (int j = 0; j < p->nu; ++j) Qd[p->nx + j] = p->r[j];
}

/* ------------------------------------------------------------------------------------------ */
/* Euclidean projections onto the input set U (textbook forms).                                */
/* ------------------------------------------------------------------------------------------ */

static int cmp_desc(const void *a, const void *b) {
  const double x = *(const double *)a, y = *(const double *)b;
  return (x < y) - (x > y);
}

int orc_project_u(const orc_problem *p, const double *y, double *out) {
  const int m = p->nu;
  const double r = p->uset_r;
  switch (p->uset) {
    case ORC_USET_BOX:
      for (int i = 0; i < m; ++i) out[i] = fmin(fmax(y[i], p->umin[i]), p->umax[i]);
      return 0;
    case ORC_USET_BALL2: {          /* y min(1, r / ||y||) */
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += y[i] * y[i];
      const double nrm = sqrt(s);
      const double f = nrm <= r ? 1.0 : r / nrm;
      for (int i = 0; i < m; ++i) out[i] = y[i] * f;
      return 0;
    }
    case ORC_USET_BALL1: {          /* soft threshold at tau (Duchi et al. 2008, sorted form) */
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += fabs(y[i]);
      if (s <= r) {
        for (int i = 0; i < m; ++i) out[i] = y[i];
        return 0;
      }
      double *a = (double *)malloc(sizeof(double) * (size_t)m);
      if (!a) return -1;
      for (int i = 0; i < m; ++i) a[i] = fabs(y[i]);
      qsort(a, (size_t)m, sizeof(double), cmp_desc);
      double run = 0.0, tau = 0.0;
      for (int j = 0; j < m; ++j) {   /* largest j with a_j - (sum_{i<=j} a_i - r) / (j+1) > 0 */
        run += a[j];
        const double t = (run - r) / (double)(j + 1);
        if (a[j] - t > 0.0) tau = t;
      }
      free(a);
      for (int i = 0; i < m; ++i) {
        const double mag = fabs(y[i]) - tau;
        out[i] = mag > 0.0 ? copysign(mag, y[i]) : 0.0;
      }
      return 0;
    }
    case ORC_USET_HALFSPACE: {      /* y - max(0, a^T y - r) / ||a||^2 a */
      double ay = 0.0, aa = 0.0;
      for (int i = 0; i < m; ++i) {
        ay += p->uset_a[i] * y[i];
        aa += p->uset_a[i] * p->uset_a[i];
      }
      const double f = ay > r ? (ay - r) / aa : 0.0;
      for (int i = 0; i < m; ++i) out[i] = y[i] - f * p->uset_a[i];
      return 0;
    }
    case ORC_USET_SOC: {            /* cone {(t, s): ||s|| <= t}, t = y_0 */
      const double t = y[0];
      double s2 = 0.0;
      for (int i = 1; i < m; ++i) s2 += y[i] * y[i];
      const double ns = sqrt(s2);
      if (ns <= t) {
        for (int i = 0; i < m; ++i) out[i] = y[i];
      } else if (ns <= -t) {
        for (int i = 0; i < m; ++i) out[i] = 0.0;
      } else {
        const double al = 0.5 * (t + ns);
        out[0] = al;
        for (int i = 1; i < m; ++i) out[i] = al * y[i] / ns;
      }
      return 0;
    }
    default:
      return -1;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Cache (Algorithm 1, "cache").                                                               */
/* ------------------------------------------------------------------------------------------ */

int orc_cache(const orc_problem *p, double *H, double *J) {
  const int nx = p->nx, nu = p->nu, n = nx + nu, N = p->N;
  const double rho = p->rho;
  double *Abar = (double *)malloc(sizeof(double) * n * n);
  double *Bbar = (double *)malloc(sizeof(double) * n * nu);
  double *ebar = (double *)malloc(sizeof(double) * n);
  double *K = (double *)malloc(sizeof(double) * n * n);
  double *AtA = (double *)malloc(sizeof(double) * n * n);
  double *Ku = (double *)malloc(sizeof(double) * nu * nu);
  double *Kuinv = (double *)malloc(sizeof(double) * nu * nu);
  double *Bt = (double *)malloc(sizeof(double) * nu * n);
  double *Qd = (double *)malloc(sizeof(double) * n);
  int rc = 0;
  if (!Abar || !Bbar || !ebar || !K || !AtA || !Ku || !Kuinv || !Bt || !Qd) { rc = -1; goto out; }
  qbar_diag(p, Qd);
  for (int k = 0; k < N; ++k) {
    /* H_k = (Qbar + rho I + rho Abar_{k+1}^T Abar_{k+1})^{-1}, or (Qbar + rho I)^{-1} at k = N-1. */
    memset(K, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) K[i * n + i] = Qd[i] + rho;
    if (k < N - 1) {
      velocity_form(nx, nu, stage_A(p, k + 1), stage_B(p, k + 1), stage_e(p, k + 1), Abar, Bbar, ebar);
      mat_tmat(n, n, n, Abar, Abar, AtA);
      for (int i = 0; i < n * n; ++i) K[i] += rho * AtA[i];
    }
    if (mat_inverse(n, K, H + (size_t)k * n * n)) { rc = -1; goto out; }
    /* J_k = (Bbar_k^T Bbar_k + W_du / rho)^{-1} Bbar_k^T. */
    velocity_form(nx, nu, stage_A(p, k), stage_B(p, k), stage_e(p, k), Abar, Bbar, ebar);
    mat_tmat(n, nu, nu, Bbar, Bbar, Ku);
    if (p->rdu)
      for (int j = 0; j < nu; ++j) Ku[j * nu + j] += p->rdu[j] / rho;
    if (mat_inverse(nu, Ku, Kuinv)) { rc = -1; goto out; }
    for (int i = 0; i < nu; ++i)
      for (int j = 0; j < n; ++j) Bt[i * n + j] = Bbar[j * nu + i];
    double *Jk = J + (size_t)k * nu * n;
    for (int i = 0; i < nu; ++i)
      for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int l = 0; l < nu; ++l) s += Kuinv[i * nu + l] * Bt[l * n + j];
        Jk[i * n + j] = s;
      }
  }
out:
  free(Abar); free(Bbar); free(ebar); free(K); free(AtA); free(Ku); free(Kuinv); free(Bt); free(Qd);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* One pass of Algorithm 1 steps 1-4.                                                          */
/* ------------------------------------------------------------------------------------------ */

int orc_iteration(const orc_problem *p, const double *H, const double *J, const double *zh,
                  const double *vh, const double *thh, const double *beh, const double *lah,
                  double *du, double *xb, double *z, double *v, double *th, double *be, double *la,
                  double *c) {
  const int nx = p->nx, nu = p->nu, n = nx + nu, N = p->N;
  const double rho = p->rho;
  double *Abar = (double *)malloc(sizeof(double) * n * n);
  double *Bbar = (double *)malloc(sizeof(double) * n * nu);
  double *ebar = (double *)malloc(sizeof(double) * n);
  double *Qd = (double *)malloc(sizeof(double) * n);
  double *t = (double *)malloc(sizeof(double) * n);
  double *y = (double *)malloc(sizeof(double) * n);
  double *Aty = (double *)malloc(sizeof(double) * n);
  double *h = (double *)malloc(sizeof(double) * n);
  double *x0b = (double *)malloc(sizeof(double) * n);
  double *ax = (double *)malloc(sizeof(double) * n);
  double *bd = (double *)malloc(sizeof(double) * n);
  double *gam = (double *)malloc(sizeof(double) * n);
  double *wv = (double *)malloc(sizeof(double) * n);
  double *zp = (double *)malloc(sizeof(double) * n);
  if (!Abar || !Bbar || !ebar || !Qd || !t || !y || !Aty || !h || !x0b || !ax || !bd || !gam ||
      !wv || !zp) {
    free(Abar); free(Bbar); free(ebar); free(Qd); free(t); free(y); free(Aty); free(h);
    free(x0b); free(ax); free(bd); free(gam); free(wv); free(zp);
    return -1;
  }
  qbar_diag(p, Qd);

  /* Step 1: for every stage k, du_k = J_k (vhat_k - betahat_k) and xbar_{k+1} = H_k h_k. */
  for (int k = 0; k < N; ++k) {
    const size_t o = (size_t)k * n;
    for (int i = 0; i < n; ++i) t[i] = vh[o + i] - beh[o + i];
    mat_vec(nu, n, J + (size_t)k * nu * n, t, du + (size_t)k * nu);
    for (int i = 0; i < n; ++i) Aty[i] = 0.0;
    if (k < N - 1) {
      /* Abar_{k+1}^T (zhat_{k+2} - vhat_{k+1} - ebar_{k+1} + lambdahat_{k+1})  [reading R2] */
      velocity_form(nx, nu, stage_A(p, k + 1), stage_B(p, k + 1), stage_e(p, k + 1), Abar, Bbar, ebar);
      const size_t o1 = (size_t)(k + 1) * n;
      for (int i = 0; i < n; ++i) y[i] = zh[o1 + i] - vh[o1 + i] - ebar[i] + lah[o1 + i];
      mat_tvec(n, n, Abar, y, Aty);
    }
    for (int i = 0; i < n; ++i) {
      double qbar_i = Qd[i] * p->ref[o + i];
      h[i] = qbar_i + rho * (zh[o + i] - thh[o + i] + Aty[i]);
    }
    mat_vec(n, n, H + (size_t)k * n * n, h, xb + o);
  }

  /* xbar_0 = col(x(t), u_prev)  [reading R6] */
  for (int i = 0; i < nx; ++i) x0b[i] = p->x0[i];
  for (int j = 0; j < nu; ++j) x0b[nx + j] = p->u_prev ? p->u_prev[j] : 0.0;

  /* Steps 2-3: closed-form (v, z) update (Theorem 1, proof form [reading R1]), then the duals. */
  double csum = 0.0;
  for (int k = 0; k < N; ++k) {
    const size_t o = (size_t)k * n;
    velocity_form(nx, nu, stage_A(p, k), stage_B(p, k), stage_e(p, k), Abar, Bbar, ebar);
    const double *xprev = (k == 0) ? x0b : xb + (size_t)(k - 1) * n;
    mat_vec(n, n, Abar, xprev, ax);                      /* Abar_k xbar_k   */
    mat_vec(n, nu, Bbar, du + (size_t)k * nu, bd);       /* Bbar_k du_k     */
    for (int i = 0; i < n; ++i) {
      gam[i] = bd[i] + beh[o + i] - ax[i] - ebar[i] + lah[o + i];
      wv[i] = (2.0 * (xb[o + i] + thh[o + i] + ax[i] + ebar[i] - lah[o + i]) + gam[i]) / 3.0;
    }
    /* z_{k+1} = Proj_Xbar(w): the box on the state part [reading R9], U on the input part
     * [reading R11]. */
    for (int i = 0; i < nx; ++i) zp[i] = fmin(fmax(wv[i], p->xmin[i]), p->xmax[i]);
    if (orc_project_u(p, wv + nx, zp + nx)) {
      free(Abar); free(Bbar); free(ebar); free(Qd); free(t); free(y); free(Aty); free(h);
      free(x0b); free(ax); free(bd); free(gam); free(wv); free(zp);
      return -1;
    }
    for (int i = 0; i < n; ++i) {
      double gamma = gam[i];
      double zi = zp[i];
      double vi = 0.5 * (zi + gamma);
      z[o + i] = zi;
      v[o + i] = vi;
      th[o + i] = thh[o + i] + xb[o + i] - zi;
      be[o + i] = beh[o + i] + bd[i] - vi;
      la[o + i] = lah[o + i] + zi - ax[i] - vi - ebar[i];   /* [reading R3] */
    }
  }
  /* Step 4: c^{i+1} = rho * sum_k of six squared norms  [readings R4, R5]. */
  for (int k = 0; k < N; ++k) {
    const size_t o = (size_t)k * n;
    for (int i = 0; i < n; ++i) {
      double dth = th[o + i] - thh[o + i];
      double dbe = be[o + i] - beh[o + i];
      double dla = la[o + i] - lah[o + i];
      double dz = z[o + i] - zh[o + i];
      double dv = v[o + i] - vh[o + i];
      double dzv = (z[o + i] - v[o + i]) - (zh[o + i] - vh[o + i]);
      csum += dth * dth + dbe * dbe + dla * dla + dz * dz + dv * dv + dzv * dzv;
    }
  }
  *c = rho * csum;
  free(Abar); free(Bbar); free(ebar); free(Qd); free(t); free(y); free(Aty); free(h);
  free(x0b); free(ax); free(bd); free(gam); free(wv); free(zp);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1 (piMPC), with the accelerated-restart steps 6-7.                                */
/* ------------------------------------------------------------------------------------------ */

int orc_solve(const orc_problem *p, const orc_options *o, double *z, double *v, double *th,
              double *be, double *la, double *du, double *xb, int *iters, double *c_final,
              int *status, double *c_hist, unsigned char *mask_hist) {
  const int nx = p->nx, nu = p->nu, n = nx + nu, N = p->N;
  const size_t sz = (size_t)N * n;
  double *H = (double *)malloc(sizeof(double) * (size_t)N * n * n);
  double *J = (double *)malloc(sizeof(double) * (size_t)N * nu * n);
  /* hats (input of the iteration), new iterates, and the previous non-hat iterates */
  double *hat = (double *)malloc(sizeof(double) * sz * 5);
  double *nw = (double *)malloc(sizeof(double) * sz * 5);
  double *cur = (double *)malloc(sizeof(double) * sz * 5);
  int rc = 0;
  if (!H || !J || !hat || !nw || !cur) { rc = -1; goto out; }
  if (orc_cache(p, H, J)) { rc = -1; goto out; }

  /* Algorithm 1 input: hat^0 = iterate^0 (e.g. from warm start); alpha_0 = 1, c^0 = 1. */
  memcpy(cur + 0 * sz, z, sizeof(double) * sz);
  memcpy(cur + 1 * sz, v, sizeof(double) * sz);
  memcpy(cur + 2 * sz, th, sizeof(double) * sz);
  memcpy(cur + 3 * sz, be, sizeof(double) * sz);
  memcpy(cur + 4 * sz, la, sizeof(double) * sz);
  memcpy(hat, cur, sizeof(double) * sz * 5);
  double alpha = 1.0, c_prev = 1.0, c = 0.0;
  int st = ORC_MAXITER, it = 0;

  for (int i = 0; i < o->max_iters; ++i) {
    if (orc_iteration(p, H, J, hat + 0 * sz, hat + 1 * sz, hat + 2 * sz, hat + 3 * sz,
                      hat + 4 * sz, du, xb, nw + 0 * sz, nw + 1 * sz, nw + 2 * sz, nw + 3 * sz,
                      nw + 4 * sz, &c)) { rc = -1; goto out; }
    it = i + 1;
    if (c_hist) c_hist[i] = c;
    if (!isfinite(c)) { st = ORC_NONFINITE; memcpy(cur, nw, sizeof(double) * sz * 5); break; }
    /* Step 5: stop on c^{i+1} <= eps; the non-hat iterates are the output. */
    if (c <= o->eps) { st = ORC_CONVERGED; memcpy(cur, nw, sizeof(double) * sz * 5); break; }
    /* Steps 6-7: momentum if c^{i+1} <= eta c^i, else restart  [reading R7]. */
    int take = 0;
    if (o->accel) take = o->force_mask ? (o->force_mask[i] != 0) : (c <= o->eta * c_prev);
    if (mask_hist) mask_hist[i] = (unsigned char)take;
    if (take) {
      double alpha_next = 0.5 + 0.5 * sqrt(1.0 + 4.0 * alpha * alpha);
      double f = (alpha - 1.0) / alpha_next;
      for (size_t j = 0; j < sz * 5; ++j) hat[j] = nw[j] + f * (nw[j] - cur[j]);
      alpha = alpha_next;
    } else {
      memcpy(hat, nw, sizeof(double) * sz * 5);
      alpha = 1.0;
    }
    memcpy(cur, nw, sizeof(double) * sz * 5);
    c_prev = c;
  }
  memcpy(z, cur + 0 * sz, sizeof(double) * sz);
  memcpy(v, cur + 1 * sz, sizeof(double) * sz);
  memcpy(th, cur + 2 * sz, sizeof(double) * sz);
  memcpy(be, cur + 3 * sz, sizeof(double) * sz);
  memcpy(la, cur + 4 * sz, sizeof(double) * sz);
  *iters = it;
  *c_final = c;
  *status = st;
out:
  free(H); free(J); free(hat); free(nw); free(cur);
  return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Nonlinear models (continuous time), written once over complex numbers so that the same     */
/* code gives f (real part at a real point) and its exact Jacobian columns by the complex-step  */
/* derivative: df/dx_j = Im f(x + i h e_j) / h.                                                */
/* ------------------------------------------------------------------------------------------ */

typedef double complex cplx;

/* Quadrotor, "+" rotor layout. x = (p[3], v[3], phi, theta, psi, w[3]), u = four rotor thrusts.
 * params = (m, g, Jx, Jy, Jz, l, k_yaw). Z-Y-X Euler angles, R = Rz(psi) Ry(theta) Rx(phi). */
static void quad_f(const double *prm, const cplx *x, const cplx *u, cplx *f) {
  const double m = prm[0], g = prm[1], Jx = prm[2], Jy = prm[3], Jz = prm[4], l = prm[5], ky = prm[6];
  cplx phi = x[6], th = x[7], psi = x[8], wx = x[9], wy = x[10], wz = x[11];
  cplx T = u[0] + u[1] + u[2] + u[3];
  cplx tx = l * (u[1] - u[3]);
  cplx ty = l * (u[2] - u[0]);
  cplx tz = ky * (u[0] - u[1] + u[2] - u[3]);
  cplx cph = ccos(phi), sph = csin(phi), cth = ccos(th), sth = csin(th), cps = ccos(psi), sps = csin(psi);
  /* third column of R: thrust direction in the world frame */
  cplx r13 = cps * sth * cph + sps * sph;
  cplx r23 = sps * sth * cph - cps * sph;
  cplx r33 = cth * cph;
  f[0] = x[3]; f[1] = x[4]; f[2] = x[5];
  f[3] = T / m * r13;
  f[4] = T / m * r23;
  f[5] = T / m * r33 - g;
  /* Euler-angle rates from body rates */
  cplx tth = sth / cth;
  f[6] = wx + sph * tth * wy + cph * tth * wz;
  f[7] = cph * wy - sph * wz;
  f[8] = (sph * wy + cph * wz) / cth;
  /* Euler's rotation equations, J diagonal */
  f[9] = (tx - (Jz - Jy) * wy * wz) / Jx;
  f[10] = (ty - (Jx - Jz) * wz * wx) / Jy;
  f[11] = (tz - (Jy - Jx) * wx * wy) / Jz;
}

/* Cart-pole (rigid pole of half-length l, frictionless), theta = 0 upright.
 * x = (pos, vel, theta, theta_dot), u = (force). params = (m_cart, m_pole, l, g). */
static void cartpole_f(const double *prm, const cplx *x, const cplx *u, cplx *f) {
  const double mc = prm[0], mp = prm[1], l = prm[2], g = prm[3];
  const double M = mc + mp;
  cplx s = csin(x[2]), c = ccos(x[2]), w = x[3];
  cplx tmp = (u[0] + mp * l * w * w * s) / M;
  cplx thacc = (g * s - c * tmp) / (l * (4.0 / 3.0 - mp * c * c / M));
  cplx xacc = tmp - mp * l * thacc * c / M;
  f[0] = x[1];
  f[1] = xacc;
  f[2] = w;
  f[3] = thacc;
}

/* CSTR of the paper's nonlinear example (Sec. V): x = (C_A, T), u = (T_c).
 * params = (C_Ai, k0, EaR, T_i). */
static void cstr_f(const double *prm, const cplx *x, const cplx *u, cplx *f) {
  const double CAi = prm[0], k0 = prm[1], EaR = prm[2], Ti = prm[3];
  cplx r = k0 * cexp(-EaR / x[1]) * x[0];
  f[0] = CAi - x[0] - r;
  f[1] = Ti + 0.3 * u[0] - 1.3 * x[1] + 11.92 * r;
}

int orc_model_dims(int model, int *nx, int *nu) {
  switch (model) {
    case ORC_MODEL_QUADROTOR: *nx = 12; *nu = 4; return 0;
    case ORC_MODEL_CARTPOLE: *nx = 4; *nu = 1; return 0;
    case ORC_MODEL_CSTR: *nx = 2; *nu = 1; return 0;
    default: return -1;
  }
}

static int model_eval(int model, const double *prm, const cplx *x, const cplx *u, cplx *f) {
  switch (model) {
    case ORC_MODEL_QUADROTOR: quad_f(prm, x, u, f); return 0;
    case ORC_MODEL_CARTPOLE: cartpole_f(prm, x, u, f); return 0;
    case ORC_MODEL_CSTR: cstr_f(prm, x, u, f); return 0;
    default: return -1;
  }
}

#define ORC_MAXDIM 32

int orc_model_f(int model, const double *params, const double *x, const double *u, double *f) {
  int nx, nu;
  if (orc_model_dims(model, &nx, &nu)) return -1;
  cplx xc[ORC_MAXDIM], uc[ORC_MAXDIM], fc[ORC_MAXDIM];
  for (int i = 0; i < nx; ++i) xc[i] = x[i];
  for (int j = 0; j < nu; ++j) uc[j] = u[j];
  if (model_eval(model, params, xc, uc, fc)) return -1;
  for (int i = 0; i < nx; ++i) f[i] = creal(fc[i]);
  return 0;
}

int orc_plant_step(int model, const double *params, double dt, const double *x, const double *u,
                   double *x_next) {
  int nx, nu;
  double f[ORC_MAXDIM];
  if (orc_model_dims(model, &nx, &nu)) return -1;
  if (orc_model_f(model, params, x, u, f)) return -1;
  for (int i = 0; i < nx; ++i) x_next[i] = x[i] + dt * f[i];
  return 0;
}

int orc_linearise(int model, const double *params, double dt, int N, const double *xbar,
                  const double *ubar, double *A, double *B, double *e) {
  int nx, nu;
  if (orc_model_dims(model, &nx, &nu)) return -1;
  const double hcs = 1e-30; /* complex-step size: exact to rounding, no cancellation */
  cplx xc[ORC_MAXDIM], uc[ORC_MAXDIM], fc[ORC_MAXDIM];
  double f0[ORC_MAXDIM];
  for (int k = 0; k < N; ++k) {
    const double *xk = xbar + (size_t)k * nx, *uk = ubar + (size_t)k * nu;
    double *Ak = A + (size_t)k * nx * nx, *Bk = B + (size_t)k * nx * nu, *ek = e + (size_t)k * nx;
    for (int i = 0; i < nx; ++i) xc[i] = xk[i];
    for (int j = 0; j < nu; ++j) uc[j] = uk[j];
    if (model_eval(model, params, xc, uc, fc)) return -1;
    for (int i = 0; i < nx; ++i) f0[i] = creal(fc[i]);
    /* A_k = I + dt df/dx */
    for (int j = 0; j < nx; ++j) {
      xc[j] = xk[j] + I * hcs;
      model_eval(model, params, xc, uc, fc);
      for (int i = 0; i < nx; ++i) Ak[i * nx + j] = (i == j ? 1.0 : 0.0) + dt * (cimag(fc[i]) / hcs);
      xc[j] = xk[j];
    }
    /* B_k = dt df/du */
    for (int j = 0; j < nu; ++j) {
      uc[j] = uk[j] + I * hcs;
      model_eval(model, params, xc, uc, fc);
      for (int i = 0; i < nx; ++i) Bk[i * nu + j] = dt * (cimag(fc[i]) / hcs);
      uc[j] = uk[j];
    }
    /* e_k = F(xbar_k, ubar_k) - A_k xbar_k - B_k ubar_k, F(x, u) = x + dt f(x, u) */
    for (int i = 0; i < nx; ++i) {
      double s = xk[i] + dt * f0[i];
      for (int j = 0; j < nx; ++j) s -= Ak[i * nx + j] * xk[j];
      for (int j = 0; j < nu; ++j) s -= Bk[i * nu + j] * uk[j];
      ek[i] = s;
    }
  }
  return 0;
}

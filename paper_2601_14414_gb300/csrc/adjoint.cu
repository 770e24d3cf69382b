// adjoint.cu -- reverse mode of the unrolled plain iteration (Algorithm 1 with hats equal to the
// iterates, a fixed number T of iterations from the zero start). The paper lists differentiating
// the solver as future work (Sec. VI); this is the derivative of the unrolled map, not of the
// optimum.
//
// One iteration maps the state S = (z, v, theta, beta, lambda) to S' (per stage k, all vectors
// of length n = nx + nu, z[k] = z_{k+1}):
//   du_k  = M_k (B_k^T t_x + t_u),  t = v_k - beta_k
//   h_k   = Qbar ref_k + rho (z_k - theta_k + Abar_{k+1}^T y_k),  y_k = z_{k+1} - v_{k+1} - ebar_{k+1} + lambda_{k+1}
//   xb_k  = H_k h_k                       (xbar_{k+1}; xbar_0 = (x0, u_prev))
//   gamma = Bbar_k du_k + beta_k - Abar_k xb_{k-1} - ebar_k + lambda_k
//   w     = (2 (xb_k + theta_k + Abar_k xb_{k-1} + ebar_k - lambda_k) + gamma) / 3
//   z'    = clamp(w, lo, hi),  v' = (z' + gamma) / 2,  theta' = theta + xb_k - z',
//   beta' = beta + Bbar_k du_k - v',  lambda' = lambda + z' - Abar_k xb_{k-1} - v' - ebar_k.
// The reverse sweep applies the transpose of each line in the opposite order. The clamp passes
// the adjoint to w when lo < w < hi, to lo when w <= lo and to hi when w >= hi. The parameters
// enter through Qbar ref_k (gradient w.r.t. ref_k: Qbar hbar_k; w.r.t. Qbar: ref_k * hbar_k),
// through H_k = (Qbar + rho I + rho Abar^T Abar)^{-1} (dH = -H dQbar H, so the Qbar gradient gains
// -hbar_k * xb_k with hbar_k = H_k xbbar_k), through xbar_0 (x0) and through the bounds.
//
// Memory. Forward states are kept every K iterations (checkpoints); the reverse sweep walks the
// segments from the last to the first, recomputes the K states of a segment from its checkpoint
// and then runs the K reverse iterations. Forward work 2T iterations, reverse T, states stored
// ceil(T/K) + K - 1 per instance.
//
// Work. One CTA per instance (largest instances first), one thread per stage (threads loop when
// N exceeds the block). All per-stage vectors live in a workspace in global memory, component
// major ([component][stage]), so that a warp's accesses to one component are coalesced; the
// stage matrices are read from the solve's stage data in any of its layouts (plain blocks:
// G with odd row stride, symmetric H and M as wrapped diagonals; blocked: H as wrapped 4 x 4
// block diagonals; halo tiles: element-major slots, H and M packed). Adjoint arithmetic runs in the iteration precision T; the per-stage
// gradient sums run in FP64. No thread waits on another CTA: only __syncthreads separates phases.
#include <algorithm>
#include <vector>

#include "launch.h"
#include "pimpc.h"
#include "solver.h"

namespace pimpc {

namespace {

constexpr int kMaxV = kMaxNLti;   // largest n any instance can have

struct AdjArgs {
  Layout L;
  const void *blk;
  const void *qd, *ref, *lo, *hi, *xb0;
  int ref_per_stage;
  double rho;
  int iters, K, nck;            // T, checkpoint spacing, number of checkpoints ceil(T / K)
  int nseg_slots;               // recompute slots per instance: max(K - 1, 2)
  const int *order;             // CTA -> instance (largest first)
  const int64_t *offT;          // per-instance workspace offset (elements of T)
  const int64_t *offD;          // per-instance accumulator offset (doubles)
  void *wsT;
  double *wsD;
  const double *dL_du, *dL_dx;  // inputs (device), may be null
  double *g_x0, *g_ref, *g_q, *g_r, *g_xmin, *g_xmax, *g_umin, *g_umax;   // outputs, may be null
};

// Per-instance views of the stage blocks and of the workspace.
template <typename T>
struct Inst {
  int nx, nu, n, N, ld, W;
  const T *blk;          // first stage block (plain) or first tile (halo tiles)
  int lti;
  int tiled, tw;         // 2: halo tiles of tw slots (W = words per tile), else plain blocks
  int oE, oH, oM;
  const T *qd, *ref, *lo, *hi, *xb0;
  int refstride;         // 0: one reference for all stages
  T rho;
  // workspace (component-major, stride N)
  T *ck;                 // nck states of 5 n N
  T *sg;                 // nseg_slots states
  T *sb;                 // adjoint state 5 n N
  T *xb, *du, *p, *yb, *xbp, *dub;
  double *hsum, *hxsum, *losum, *hisum, *gx0;

  // Stage k's block: element e at slot(k)[e * es()].
  __device__ const T *slot(int k) const {
    if (tiled == 2) {
      int t, sl;
      halo_slot(tw, k, t, sl);
      return blk + (int64_t)t * W + sl;
    }
    return blk + (lti ? 0 : (int64_t)k * W);
  }
  __device__ int es() const { return tiled == 2 ? tw : 1; }
  // G_k(r, c), e_k(r), H_k(r, c), M_k(r, c) in any layout (plain and blocked: G rows of stride
  // ld, M as wrapped diagonals, H as wrapped diagonals or wrapped 4 x 4 block diagonals; halo
  // tiles: G row-major, H and M packed lower).
  __device__ T Gv(int k, int r, int c) const {
    return tiled == 2 ? slot(k)[(r * n + c) * tw] : slot(k)[r * ld + c];
  }
  __device__ T Ev(int k, int r) const {
    return tiled == 2 ? slot(k)[(nx * n + r) * tw] : slot(k)[oE + r];
  }
  __device__ T Hv(int k, int r, int c) const;
  __device__ T Mv(int k, int r, int c) const;
  __device__ T *st(T *base, int b, int c) const { return base + (int64_t)(b * n + c) * N; }
  __device__ const T *cst(const T *base, int b, int c) const {
    return base + (int64_t)(b * n + c) * N;
  }
  __device__ const T *refk(int k) const { return ref ? ref + (int64_t)refstride * k : nullptr; }
};

// Element (r, c) of a symmetric m x m matrix stored as wrapped diagonals (row d holds
// S[c][(c + d) mod m] for d <= m / 2).
template <typename T>
__device__ __forceinline__ T sym_at(const T *Wp, int m, int r, int c) {
  int d = c - r;
  if (d < 0) d += m;
  return (2 * d <= m) ? Wp[d * m + r] : Wp[(m - d) * m + c];
}

// Element (r, c) of a symmetric m x m matrix stored as wrapped 4 x 4 block diagonals (block
// (d, I) = S_{I, (I+d) mod nb} for d <= nb / 2; the middle diagonal of an even nb only for
// I < nb / 2; the diagonal blocks d = 0 only their upper triangles).
template <typename T>
__device__ __forceinline__ T sym_block_at(const T *Hb, int m, int r, int c) {
  const int nb = bl_nb(m);
  int I = r >> 2, a = r & 3, J = c >> 2, b = c & 3;
  int d = J - I;
  if (d < 0) d += nb;
  if (2 * d > nb || (2 * d == nb && I >= (nb >> 1)) || (d == 0 && a > b)) {
    // stored as the transpose: block (nb - d, J) (the middle diagonal of an even nb: block row
    // J = I - nb/2; a diagonal block: its upper triangle), element (b, a)
    d = d == 0 ? 0 : nb - d;
    int t = I; I = J; J = t;
    t = a; a = b; b = t;
  }
  return Hb[bl_sym_index(nb, d, I, a, b)];
}

template <typename T>
__device__ T Inst<T>::Hv(int k, int r, int c) const {
  if (tiled == 2) {
    const int i = r > c ? r : c, q = r > c ? c : r;
    return slot(k)[(nx * n + nx + i * (i + 1) / 2 + q) * tw];
  }
  const T *b = blk + (lti ? ((k < N - 1) ? 0 : W) : (int64_t)k * W) + oH;
  return tiled == 3 ? sym_block_at(b, n, r, c) : sym_at(b, n, r, c);
}

template <typename T>
__device__ T Inst<T>::Mv(int k, int r, int c) const {
  if (tiled == 2) {
    const int i = r > c ? r : c, q = r > c ? c : r;
    return slot(k)[(nx * n + nx + n * (n + 1) / 2 + i * (i + 1) / 2 + q) * tw];
  }
  return sym_at(slot(k) + oM, nu, r, c);
}

template <typename T>
__device__ void make_inst(const AdjArgs &a, int j, Inst<T> &I) {
  I.nx = a.L.nx[j];
  I.nu = a.L.nu[j];
  I.n = I.nx + I.nu;
  I.N = a.L.N[j];
  const int ts = (int)sizeof(T);
  I.ld = a.L.tiled == 3 ? bl_ldg(I.n, ts) : odd_ld(I.n);
  I.W = a.L.W[j];
  I.lti = a.L.lti;
  I.tiled = a.L.tiled;
  I.tw = a.L.tiled == 2 ? a.L.tw[j] : 0;
  I.blk = (const T *)a.blk + a.L.blk[j];
  I.oE = I.nx * I.ld;
  I.oH = a.L.tiled == 3 ? bl_oH(I.nx, I.nu, ts) : I.oE + I.nx;
  I.oM = a.L.tiled == 3 ? bl_oM(I.nx, I.nu, ts) : I.oH + wrapped_size(I.n);
  I.qd = (const T *)a.qd + a.L.off_n[j];
  I.ref = a.ref ? (const T *)a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j]) : nullptr;
  I.refstride = a.ref_per_stage ? I.n : 0;
  I.lo = (const T *)a.lo + a.L.off_n[j];
  I.hi = (const T *)a.hi + a.L.off_n[j];
  I.xb0 = (const T *)a.xb0 + a.L.off_n[j];
  I.rho = (T)a.rho;
  const int64_t sN = (int64_t)5 * I.n * I.N;
  T *w = (T *)a.wsT + a.offT[j];
  I.ck = w;
  I.sg = I.ck + (int64_t)a.nck * sN;
  I.sb = I.sg + (int64_t)a.nseg_slots * sN;
  I.xb = I.sb + sN;
  I.du = I.xb + (int64_t)I.n * I.N;
  I.p = I.du + (int64_t)I.nu * I.N;
  I.yb = I.p + (int64_t)I.n * I.N;
  I.xbp = I.yb + (int64_t)I.n * I.N;
  I.dub = I.xbp + (int64_t)I.n * I.N;
  double *d = a.wsD + a.offD[j];
  I.hsum = d;
  I.hxsum = d + (int64_t)I.n * I.N;
  I.losum = d + (int64_t)2 * I.n * I.N;
  I.hisum = d + (int64_t)3 * I.n * I.N;
  I.gx0 = d + (int64_t)4 * I.n * I.N;
}

// ---- forward, first half: du_k and xb_k of every stage (Algorithm 1 step 1) ---------------
template <typename T>
__device__ void fwd_step1(const Inst<T> &I, const T *S) {
  const int nx = I.nx, nu = I.nu, n = I.n, N = I.N;
  T t[kMaxV], h[kMaxV];
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    for (int c = 0; c < n; ++c) t[c] = I.cst(S, 1, c)[k] - I.cst(S, 3, c)[k];
    // w = B_k^T t_x + t_u, du = M_k w
    T w[kMaxV];
    for (int q = 0; q < nu; ++q) {
      T s = t[nx + q];
      for (int r = 0; r < nx; ++r) s += I.Gv(k, r, nx + q) * t[r];
      w[q] = s;
    }
    for (int q = 0; q < nu; ++q) {
      T s = (T)0;
      for (int i = 0; i < nu; ++i) s += I.Mv(k, q, i) * w[i];
      I.du[(int64_t)q * N + k] = s;
    }
    // h = Qbar ref_k + rho (z_k - theta_k + Abar_{k+1}^T y_k)
    for (int c = 0; c < n; ++c) h[c] = (T)0;
    if (k < N - 1) {
      T y[kMaxV];
      for (int c = 0; c < n; ++c)
        y[c] = I.cst(S, 0, c)[k + 1] - I.cst(S, 1, c)[k + 1] + I.cst(S, 4, c)[k + 1] -
               (c < nx ? I.Ev(k + 1, c) : (T)0);
      for (int c = 0; c < n; ++c) {
        T s = c < nx ? (T)0 : y[c];
        for (int r = 0; r < nx; ++r) s += I.Gv(k + 1, r, c) * y[r];
        h[c] = s;
      }
    }
    const T *rf = I.refk(k);
    for (int c = 0; c < n; ++c)
      h[c] = I.qd[c] * (rf ? rf[c] : (T)0) + I.rho * (I.cst(S, 0, c)[k] - I.cst(S, 2, c)[k] + h[c]);
    for (int r = 0; r < n; ++r) {
      T s = (T)0;
      for (int c = 0; c < n; ++c) s += I.Hv(k, r, c) * h[c];
      I.xb[(int64_t)r * N + k] = s;
    }
  }
}

// Abar_k xb_{k-1} (ax), Bbar_k du_k (bd) and ebar_k (ee) of stage k.
template <typename T>
__device__ __forceinline__ void stage_products(const Inst<T> &I, int k, T *ax, T *bd, T *ee) {
  const int nx = I.nx, nu = I.nu, n = I.n, N = I.N;
  T xp[kMaxV];
  for (int c = 0; c < n; ++c) xp[c] = k == 0 ? I.xb0[c] : I.xb[(int64_t)c * N + k - 1];
  for (int r = 0; r < nx; ++r) {
    T s = (T)0;
    for (int c = 0; c < n; ++c) s += I.Gv(k, r, c) * xp[c];
    ax[r] = s;
    T b = (T)0;
    for (int q = 0; q < nu; ++q) b += I.Gv(k, r, nx + q) * I.du[(int64_t)q * N + k];
    bd[r] = b;
    ee[r] = I.Ev(k, r);
  }
  for (int q = 0; q < nu; ++q) {
    ax[nx + q] = xp[nx + q];
    bd[nx + q] = I.du[(int64_t)q * N + k];
    ee[nx + q] = (T)0;
  }
}

// ---- forward, second half: steps 2-3, S -> Sout ---------------------------------------------
template <typename T>
__device__ void fwd_step23(const Inst<T> &I, const T *S, T *Sout) {
  const int n = I.n, N = I.N;
  T ax[kMaxV], bd[kMaxV], ee[kMaxV];
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    stage_products(I, k, ax, bd, ee);
    for (int c = 0; c < n; ++c) {
      const T be = I.cst(S, 3, c)[k], la = I.cst(S, 4, c)[k], th = I.cst(S, 2, c)[k];
      const T x1 = I.xb[(int64_t)c * N + k];
      const T gam = bd[c] + be - ax[c] - ee[c] + la;
      const T w = ((T)2 * (x1 + th + ax[c] + ee[c] - la) + gam) / (T)3;
      const T lo = I.lo[c], hi = I.hi[c];
      const T z = w < lo ? lo : (w > hi ? hi : w);
      const T v = (T)0.5 * (z + gam);
      I.st(Sout, 0, c)[k] = z;
      I.st(Sout, 1, c)[k] = v;
      I.st(Sout, 2, c)[k] = th + x1 - z;
      I.st(Sout, 3, c)[k] = be + bd[c] - v;
      I.st(Sout, 4, c)[k] = la + z - ax[c] - v - ee[c];
    }
  }
}

// ---- reverse of steps 2-3 (and the neighbour term of the previous reverse step 1) ----------
template <typename T>
__device__ void rev_step23(const Inst<T> &I, const T *S) {
  const int nx = I.nx, nu = I.nu, n = I.n, N = I.N;
  T ax[kMaxV], bd[kMaxV], ee[kMaxV], axb[kMaxV], bdb[kMaxV];
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    // Adjoint of y_{k-1} = z_k - v_k - ebar_k + lambda_k, left by the later reverse step 1.
    if (k > 0)
      for (int c = 0; c < n; ++c) {
        const T yb = I.yb[(int64_t)c * N + k - 1];
        I.st(I.sb, 0, c)[k] += yb;
        I.st(I.sb, 1, c)[k] -= yb;
        I.st(I.sb, 4, c)[k] += yb;
      }
    stage_products(I, k, ax, bd, ee);
    for (int c = 0; c < n; ++c) {
      const T be = I.cst(S, 3, c)[k], la = I.cst(S, 4, c)[k], th = I.cst(S, 2, c)[k];
      const T x1 = I.xb[(int64_t)c * N + k];
      const T gam = bd[c] + be - ax[c] - ee[c] + la;
      const T w = ((T)2 * (x1 + th + ax[c] + ee[c] - la) + gam) / (T)3;
      const T lo = I.lo[c], hi = I.hi[c];
      const T zb = I.st(I.sb, 0, c)[k], vb = I.st(I.sb, 1, c)[k], thb = I.st(I.sb, 2, c)[k];
      const T beb = I.st(I.sb, 3, c)[k], lab = I.st(I.sb, 4, c)[k];
      const T vt = vb - lab - beb;                  // adjoint of v' (all uses)
      const T zt = zb + lab - thb + (T)0.5 * vt;    // adjoint of z' (all uses)
      T wb = (T)0;
      if (w <= lo) I.losum[(int64_t)c * N + k] += (double)zt;
      else if (w >= hi) I.hisum[(int64_t)c * N + k] += (double)zt;
      else wb = zt;
      const T gb = (T)0.5 * vt + wb / (T)3;         // adjoint of gamma
      const T w23 = (T)2 * wb / (T)3;
      axb[c] = -lab + w23 - gb;
      bdb[c] = beb + gb;
      I.xbp[(int64_t)c * N + k] = thb + w23;
      I.st(I.sb, 0, c)[k] = (T)0;
      I.st(I.sb, 1, c)[k] = (T)0;
      I.st(I.sb, 2, c)[k] = thb + w23;
      I.st(I.sb, 3, c)[k] = beb + gb;
      I.st(I.sb, 4, c)[k] = lab - w23 + gb;
    }
    // dubar = Bbar_k^T bdbar
    for (int q = 0; q < nu; ++q) {
      T s = bdb[nx + q];
      for (int r = 0; r < nx; ++r) s += I.Gv(k, r, nx + q) * bdb[r];
      I.dub[(int64_t)q * N + k] = s;
    }
    // Abar_k^T axbar: to xb_{k-1} (read by the thread of stage k-1), or to xbar_0 = (x0, u_prev).
    for (int c = 0; c < n; ++c) {
      T s = c < nx ? (T)0 : axb[c];
      for (int r = 0; r < nx; ++r) s += I.Gv(k, r, c) * axb[r];
      if (k > 0) I.p[(int64_t)c * N + k] = s;
      else if (c < nx) I.gx0[c] += (double)s;
    }
  }
}

// ---- reverse of step 1 -----------------------------------------------------------------------
template <typename T>
__device__ void rev_step1(const Inst<T> &I) {
  const int nx = I.nx, nu = I.nu, n = I.n, N = I.N;
  T xt[kMaxV], hb[kMaxV], m[kMaxV];
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    for (int c = 0; c < n; ++c)
      xt[c] = I.xbp[(int64_t)c * N + k] + (k < N - 1 ? I.p[(int64_t)c * N + k + 1] : (T)0);
    for (int r = 0; r < n; ++r) {
      T s = (T)0;
      for (int c = 0; c < n; ++c) s += I.Hv(k, r, c) * xt[c];
      hb[r] = s;
    }
    for (int c = 0; c < n; ++c) {
      I.hsum[(int64_t)c * N + k] += (double)hb[c];
      I.hxsum[(int64_t)c * N + k] += (double)hb[c] * (double)I.xb[(int64_t)c * N + k];
      I.st(I.sb, 0, c)[k] += I.rho * hb[c];
      I.st(I.sb, 2, c)[k] -= I.rho * hb[c];
    }
    if (k < N - 1) {
      // ybar = Abar_{k+1} (rho hbar): [A x_x + B x_u ; x_u]
      for (int r = 0; r < nx; ++r) {
        T s = (T)0;
        for (int c = 0; c < n; ++c) s += I.Gv(k + 1, r, c) * (I.rho * hb[c]);
        I.yb[(int64_t)r * N + k] = s;
      }
      for (int q = 0; q < nu; ++q) I.yb[(int64_t)(nx + q) * N + k] = I.rho * hb[nx + q];
    }
    // tbar = Bbar_k M_k dubar -> v_k (+), beta_k (-)
    for (int q = 0; q < nu; ++q) {
      T s = (T)0;
      for (int i = 0; i < nu; ++i) s += I.Mv(k, q, i) * I.dub[(int64_t)i * N + k];
      m[q] = s;
    }
    for (int r = 0; r < nx; ++r) {
      T s = (T)0;
      for (int q = 0; q < nu; ++q) s += I.Gv(k, r, nx + q) * m[q];
      I.st(I.sb, 1, r)[k] += s;
      I.st(I.sb, 3, r)[k] -= s;
    }
    for (int q = 0; q < nu; ++q) {
      I.st(I.sb, 1, nx + q)[k] += m[q];
      I.st(I.sb, 3, nx + q)[k] -= m[q];
    }
  }
}

template <typename T>
__device__ void zero_state(const Inst<T> &I, T *S, int comps) {
  const int64_t cnt = (int64_t)comps * I.N;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) S[i] = (T)0;
}

template <typename T>
__global__ void __launch_bounds__(256) adjoint_kernel(AdjArgs a) {
  const int j = a.order[blockIdx.x];
  Inst<T> I;
  make_inst(a, j, I);
  const int n = I.n, N = I.N, nx = I.nx;
  const int64_t sN = (int64_t)5 * n * N;
  const int Tn = a.iters, K = a.K;

  // Zero start, accumulators, neighbour buffers.
  zero_state(I, I.ck, 5 * n);
  zero_state(I, I.yb, n);
  zero_state(I, I.p, n);
  for (int64_t i = threadIdx.x; i < (int64_t)4 * n * N + nx; i += blockDim.x) I.hsum[i] = 0.0;
  // Adjoint of the last iterate: z[k] = (x_{k+1}, u_k).
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    for (int c = 0; c < 5 * n; ++c) {
      T g = (T)0;
      if (c < nx) g = a.dL_dx ? (T)a.dL_dx[a.L.Nnx[j] + (int64_t)k * nx + c] : (T)0;
      else if (c < n) g = a.dL_du ? (T)a.dL_du[a.L.Nnu[j] + (int64_t)k * I.nu + c - nx] : (T)0;
      I.sb[(int64_t)c * N + k] = g;
    }
  __syncthreads();

  // Forward sweep: checkpoints at iterations 0, K, 2K, ...
  {
    const T *cur = I.ck;
    int ping = 0;
    for (int i = 0; i < (a.nck - 1) * K; ++i) {
      T *out = ((i + 1) % K == 0) ? I.ck + (int64_t)((i + 1) / K) * sN : I.sg + (int64_t)ping * sN;
      if ((i + 1) % K != 0) ping ^= 1;
      fwd_step1(I, cur);
      __syncthreads();
      fwd_step23(I, cur, out);
      __syncthreads();
      cur = out;
    }
  }

  // Reverse sweep, segment by segment.
  for (int seg = a.nck - 1; seg >= 0; --seg) {
    const int start = seg * K;
    const int len = min(K, Tn - start);
    auto state = [&](int m) -> T * { return m == 0 ? I.ck + (int64_t)seg * sN : I.sg + (int64_t)(m - 1) * sN; };
    for (int m = 0; m + 1 < len; ++m) {
      fwd_step1(I, state(m));
      __syncthreads();
      fwd_step23(I, state(m), state(m + 1));
      __syncthreads();
    }
    for (int m = len - 1; m >= 0; --m) {
      const T *S = state(m);
      fwd_step1(I, S);              // xb, du of this iteration
      __syncthreads();
      rev_step23(I, S);
      __syncthreads();
      rev_step1(I);
      __syncthreads();
    }
  }

  // Gradients of this instance (sums over stages in stage order).
  const int nu = I.nu;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double gq = 0.0, glo = 0.0, ghi = 0.0, gref = 0.0;
    const double qd = (double)I.qd[c];
    for (int k = 0; k < N; ++k) {
      const int64_t o = (int64_t)c * N + k;
      const T *rf = I.refk(k);
      const double rv = rf ? (double)rf[c] : 0.0;
      gq += rv * I.hsum[o] - I.hxsum[o];
      glo += I.losum[o];
      ghi += I.hisum[o];
      gref += qd * I.hsum[o];
      if (a.g_ref && a.ref_per_stage) a.g_ref[a.L.Nn[j] + (int64_t)k * n + c] = qd * I.hsum[o];
    }
    if (a.g_ref && !a.ref_per_stage) a.g_ref[a.L.off_n[j] + c] = gref;
    if (c < nx) {
      if (a.g_q) a.g_q[a.L.off_nx[j] + c] = gq;
      if (a.g_xmin) a.g_xmin[a.L.off_nx[j] + c] = glo;
      if (a.g_xmax) a.g_xmax[a.L.off_nx[j] + c] = ghi;
      if (a.g_x0) a.g_x0[a.L.off_nx[j] + c] = I.gx0[c];
    } else {
      const int q = c - nx;
      if (a.g_r) a.g_r[a.L.off_nu[j] + q] = gq;
      if (a.g_umin) a.g_umin[a.L.off_nu[j] + q] = glo;
      if (a.g_umax) a.g_umax[a.L.off_nu[j] + q] = ghi;
    }
  }
  (void)nu;
}

}  // namespace

}  // namespace pimpc

using namespace pimpc;

extern "C" int pimpc_backward(pimpc_solver *s, const double *dL_du, const double *dL_dx,
                              double *g_x0, double *g_ref, double *g_q, double *g_r,
                              double *g_xmin, double *g_xmax, double *g_umin, double *g_umax,
                              int checkpoint_every, int mem, void *stream) {
  if (!s) return PIMPC_EINVAL;
  if (mem != PIMPC_HOST && mem != PIMPC_DEVICE) return fail(s, PIMPC_EINVAL, "bad mem");
  if (checkpoint_every < 1) return fail(s, PIMPC_EINVAL, "checkpoint_every must be >= 1");
  if (!s->solved) return fail(s, PIMPC_ESTATE, "no solve has run");
  if (s->last_polished)
    return fail(s, PIMPC_ESTATE, "the last solve ran an FP64 polish; the adjoint covers one precision");
  if (s->last_warm != 0 || s->last_accel != 0 || s->last_eps >= 0.0)
    return fail(s, PIMPC_ESTATE,
                "the last solve must use warm_start = 0, accel = 0 and eps < 0 (fixed iterations)");
  if (s->tiled == 1 || s->tiled == 4)
    return fail(s, PIMPC_ESTATE, "the adjoint does not read the tiled iterate layouts (schedules 6 and the static entry point)");
  if (s->any_uset) return fail(s, PIMPC_ESTATE, "the adjoint covers box input sets only");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  const int Tn = s->last_iters_fixed;
  const int K = std::min(checkpoint_every, std::max(Tn, 1));
  const int nck = (Tn + K - 1) / K;
  const int slots = std::max(K - 1, 2);
  const size_t ts = tsize(s->prec);

  // Workspace: per-instance T region and FP64 accumulators, the CTA order, host staging.
  std::vector<int64_t> offT(s->batch), offD(s->batch);
  int64_t totT = 0, totD = 0;
  int maxN = 1;
  for (int j = 0; j < s->batch; ++j) {
    const int64_t n = s->nx[j] + s->nu[j], N = s->N[j], nu = s->nu[j];
    offT[j] = totT;
    // checkpoints, recompute slots and the adjoint state (5 n N each); xb, p, yb, xbp (n N);
    // du, dubar (nu N)
    totT += (5 * n * N) * (nck + slots + 1) + 4 * n * N + 2 * nu * N;
    totT = (totT + 31) & ~(int64_t)31;
    offD[j] = totD;
    totD += 4 * n * N + s->nx[j];
    totD = (totD + 3) & ~(int64_t)3;
    maxN = std::max(maxN, (int)N);
  }
  const int64_t n_ref = s->last_ref_per_stage ? s->tot_Nn : s->tot_n;
  const int64_t stage_in = s->tot_Nnu + s->tot_Nnx;
  const int64_t stage_out = 3 * s->tot_nx + 3 * s->tot_nu + s->tot_nx + n_ref;
  auto rounded = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t parts[7] = {sizeof(int64_t) * s->batch, sizeof(int64_t) * s->batch,
                           sizeof(int) * s->batch,     sizeof(double) * totD,
                           sizeof(double) * stage_in,  sizeof(double) * stage_out,
                           ts * totT};
  size_t bytes = 0;
  for (size_t b : parts) bytes += rounded(b);
  if (bytes > s->adj_ws_bytes) {
    if (s->adj_ws) {
      cudaStreamSynchronize(st);
      cudaFree(s->adj_ws);
      s->adj_ws = nullptr;
      s->adj_ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&s->adj_ws, bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      s->adj_ws = nullptr;
      return fail(s, e == cudaErrorMemoryAllocation ? PIMPC_ENOMEM : PIMPC_ECUDA,
                  std::string("adjoint workspace: ") + cudaGetErrorString(e));
    }
    s->adj_ws_bytes = bytes;
  }
  char *w = (char *)s->adj_ws;
  int pi = 0;
  auto carve = [&]() { char *p = w; w += rounded(parts[pi++]); return p; };
  int64_t *d_offT = (int64_t *)carve();
  int64_t *d_offD = (int64_t *)carve();
  int *d_order = (int *)carve();
  double *d_acc = (double *)carve();
  double *d_in = (double *)carve();
  double *d_out = (double *)carve();
  void *d_T = carve();

  std::vector<int> order(s->batch);
  for (int j = 0; j < s->batch; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const double cx = (double)s->N[x] * (s->nx[x] + s->nu[x]) * (s->nx[x] + s->nu[x]);
    const double cy = (double)s->N[y] * (s->nx[y] + s->nu[y]) * (s->nx[y] + s->nu[y]);
    return cx > cy;
  });
  PIMPC_CHECK(s, cudaMemcpyAsync(d_offT, offT.data(), sizeof(int64_t) * s->batch, cudaMemcpyHostToDevice, st), "adjoint offsets");
  PIMPC_CHECK(s, cudaMemcpyAsync(d_offD, offD.data(), sizeof(int64_t) * s->batch, cudaMemcpyHostToDevice, st), "adjoint offsets");
  PIMPC_CHECK(s, cudaMemcpyAsync(d_order, order.data(), sizeof(int) * s->batch, cudaMemcpyHostToDevice, st), "adjoint order");

  AdjArgs a{};
  a.L = s->L;
  a.blk = s->blk_T;
  a.qd = s->qd_T;
  a.ref = s->last_ref_given ? s->ref_T : nullptr;
  a.ref_per_stage = s->last_ref_per_stage;
  a.lo = s->lo_T;
  a.hi = s->hi_T;
  a.xb0 = s->xb0_T;
  a.rho = s->rho;
  a.iters = Tn;
  a.K = K;
  a.nck = nck;
  a.nseg_slots = slots;
  a.order = d_order;
  a.offT = d_offT;
  a.offD = d_offD;
  a.wsT = d_T;
  a.wsD = d_acc;
  const bool host = mem == PIMPC_HOST;
  if (host) {
    if (dL_du) PIMPC_CHECK(s, cudaMemcpyAsync(d_in, dL_du, sizeof(double) * s->tot_Nnu, cudaMemcpyHostToDevice, st), "copy dL_du");
    if (dL_dx) PIMPC_CHECK(s, cudaMemcpyAsync(d_in + s->tot_Nnu, dL_dx, sizeof(double) * s->tot_Nnx, cudaMemcpyHostToDevice, st), "copy dL_dx");
    a.dL_du = dL_du ? d_in : nullptr;
    a.dL_dx = dL_dx ? d_in + s->tot_Nnu : nullptr;
    double *o = d_out;
    auto slot = [&](double *user, int64_t cnt) { double *p = user ? o : nullptr; o += cnt; return p; };
    a.g_x0 = slot(g_x0, s->tot_nx);
    a.g_q = slot(g_q, s->tot_nx);
    a.g_xmin = slot(g_xmin, s->tot_nx);
    a.g_xmax = slot(g_xmax, s->tot_nx);
    a.g_r = slot(g_r, s->tot_nu);
    a.g_umin = slot(g_umin, s->tot_nu);
    a.g_umax = slot(g_umax, s->tot_nu);
    a.g_ref = slot(g_ref, n_ref);
  } else {
    a.dL_du = dL_du;
    a.dL_dx = dL_dx;
    a.g_x0 = g_x0; a.g_q = g_q; a.g_xmin = g_xmin; a.g_xmax = g_xmax;
    a.g_r = g_r; a.g_umin = g_umin; a.g_umax = g_umax; a.g_ref = g_ref;
  }
  const int threads = std::min(256, std::max(32, (maxN + 31) / 32 * 32));
  if (s->prec == PIMPC_F32) adjoint_kernel<float><<<s->batch, threads, 0, st>>>(a);
  else adjoint_kernel<double><<<s->batch, threads, 0, st>>>(a);
  PIMPC_CHECK(s, cudaGetLastError(), "adjoint launch");
  if (host) {
    struct { double *user, *dev; int64_t cnt; } outs[8] = {
        {g_x0, a.g_x0, s->tot_nx}, {g_q, a.g_q, s->tot_nx}, {g_xmin, a.g_xmin, s->tot_nx},
        {g_xmax, a.g_xmax, s->tot_nx}, {g_r, a.g_r, s->tot_nu}, {g_umin, a.g_umin, s->tot_nu},
        {g_umax, a.g_umax, s->tot_nu}, {g_ref, a.g_ref, n_ref}};
    for (auto &o : outs)
      if (o.user) PIMPC_CHECK(s, cudaMemcpyAsync(o.user, o.dev, sizeof(double) * o.cnt, cudaMemcpyDeviceToHost, st), "copy gradient");
    PIMPC_CHECK(s, cudaStreamSynchronize(st), "backward");
  }
  return PIMPC_OK;
}

// factorise.cu -- the per-stage cache of Algorithm 1 ("cache J_k and H_k"), computed in FP64.
//
// For stage k (LTV) the warp forms
//   K = Qbar + rho I + rho Abar_{k+1}^T Abar_{k+1}   (k < N-1),   K = Qbar + rho I   (k = N-1),
// where Abar^T Abar = G^T G + diag(0, I_nu) with G = [A | B] (Theorem 2's velocity form), and
// writes H_k = K^{-1}, inverted by sweeps of the symmetric matrix (Gauss-Jordan elimination in
// pivot order, which needs no pivoting for a positive definite K). It also writes
// M_k = (B_k^T B_k + I + Wdu / rho)^{-1}, so that the du update of Algorithm 1 step 1,
// J_k (v - beta) with J_k = (Bbar^T Bbar)^{-1} Bbar^T, is M_k (B_k^T (v - beta)_x + (v - beta)_u);
// and it copies G_k and e_k into the stage block.
// Outputs are converted to the iteration precision T. LTI instances have two blocks: block 0
// with H = (Qbar + rho I + rho Abar^T Abar)^{-1} and block 1 with the terminal H_{N-1}.
#include "bl_slot.cuh"
#include "launch.h"

namespace pimpc {

namespace {

struct FactArgs {
  Layout L;
  const double *A, *B, *e;   // FP64 dynamics, user layout
  const double *qd;          // [sum n] Qbar diagonal in FP64
  const double *rdu;         // [sum n] with the W_du diagonal at the input slots (or null)
  double rho;
  const int *binst;          // instance of each global block
  const int64_t *bbase;      // first global block of each instance
  int64_t nblocks;
  int words_per_warp;        // shared-memory doubles per warp
  int *err;                  // [batch]: set to 1 for an instance with a non-positive pivot
};

// Row i and column c <= i of the t-th lower-triangle entry in row-major order
// (t = i (i + 1) / 2 + c), so that a warp's lanes take consecutive entries.
__device__ __forceinline__ void tri_index(int t, int &i, int &c) {
  i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  c = t - i * (i + 1) / 2;
}

// The inverse of the symmetric positive definite m x m matrix whose lower triangle is in S
// (row-major, leading dimension ld), by m sweeps of the symmetric matrix (Gauss-Jordan
// elimination with the pivots in order; for a positive definite matrix every pivot is positive,
// and a pivot that is not flags err): sweeping pivot k with d = 1 / a_kk sets a_ij -= a_ik a_kj d
// for i, j != k, a_ik = a_ik d, a_kk = -d; after all m sweeps the matrix holds -S^{-1}. The lanes
// share the entries of the lower triangle (t = lane, lane + 32, ... in row-major order), so that
// every FP64 instruction of a sweep has all 32 lanes busy. X (m x m, leading dimension ld)
// serves as scratch for the pivot column during the sweeps and receives S^{-1} (both triangles).
__device__ void sweep_inverse(double *S, double *X, int m, int ld, int lane, int *err) {
  double *col = X, *cold = X + m;  // column k, and column k times d
  const int T = m * (m + 1) / 2;
  int i0 = 0, j0 = 0;
  if (lane < T) tri_index(lane, i0, j0);
  for (int k = 0; k < m; ++k) {
    __syncwarp();
    double akk = S[k * ld + k];
    if (!(akk > 0.0)) {
      if (lane == 0) *err = 1;
      akk = 1.0;
    }
    const double d = 1.0 / akk;
    for (int i = lane; i < m; i += 32) {
      const double c = i >= k ? S[i * ld + k] : S[k * ld + i];
      col[i] = c;
      cold[i] = c * d;
    }
    __syncwarp();
    int i = i0, j = j0;
    for (int t = lane; t < T; t += 32) {
      double v;
      if (i == k) v = (j == k) ? -d : cold[j];
      else if (j == k) v = cold[i];
      else v = fma(-col[i], cold[j], S[i * ld + j]);
      S[i * ld + j] = v;
      j += 32;  // the entry 32 further on in row-major order
      while (j > i) { j -= i + 1; ++i; }
    }
  }
  __syncwarp();
  for (int t = lane; t < m * m; t += 32) {
    const int r = t / m, c = t - r * m;
    X[r * ld + c] = -(r >= c ? S[r * ld + c] : S[c * ld + r]);
  }
  __syncwarp();
}

template <typename T>
__global__ void factorise_kernel(FactArgs a, T *blk) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= a.nblocks) return;
  double *sh = smem + (size_t)warp * a.words_per_warp;
  const int j = a.binst[b];
  const int kb = (int)(b - a.bbase[j]);
  const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
  const int ld = n;
  double *G = sh;                    // nx x n
  double *S = G + nx * n;            // n x n  (K, then L)
  double *X = S + n * n;             // n x n  (inverse)
  const bool lti = a.L.lti != 0;
  const bool terminal = lti ? (kb == 1) : (kb == N - 1);
  const double rho = a.rho;
  const double *qd = a.qd + a.L.off_n[j];

  // Dynamics of the stage whose Abar enters H (k+1), and of the stage itself (k).
  const int kH = lti ? 0 : kb + 1;
  const int kS = lti ? 0 : kb;
  const double *A = a.A + a.L.offA[j];
  const double *B = a.B + a.L.offB[j];
  const double *e = a.e ? a.e + a.L.offe[j] : nullptr;

  // K = Qbar + rho I (+ rho (G^T G + diag(0, I))), lower triangle.
  if (!terminal) {
    const double *Ak = A + (size_t)kH * nx * nx, *Bk = B + (size_t)kH * nx * nu;
    for (int w = lane; w < nx * n; w += 32) {
      int r = w / n, c = w - r * n;
      G[w] = c < nx ? Ak[r * nx + c] : Bk[r * nu + (c - nx)];
    }
  }
  __syncwarp();
  for (int t = lane; t < n * (n + 1) / 2; t += 32) {  // every lane its own (i, c), c <= i
    int i, c;
    tri_index(t, i, c);
    double s = 0.0;
    if (!terminal) {
      for (int r = 0; r < nx; ++r) s += G[r * n + i] * G[r * n + c];
      if (i == c && i >= nx) s += 1.0;
    }
    s *= rho;
    if (i == c) s += qd[i] + rho;
    S[i * ld + c] = s;
  }
  sweep_inverse(S, X, n, ld, lane, a.err + j);

  const int W = a.L.W[j];
  const int lay = a.L.tiled;
  const bool packed = lay == 1 || lay == 2;  // symmetric matrices packed lower
  const bool blocked = lay == 3;
  const int ts = (int)sizeof(T);
  const int ldg = blocked ? bl_ldg(n, ts) : (packed ? n : odd_ld(n));
  const int oE = nx * ldg;
  const int oH = blocked ? bl_oH(nx, nu, ts) : oE + nx;
  const int oM = blocked ? bl_oM(nx, nu, ts) : oH + (packed ? packed_size(n) : wrapped_size(n));
  // Element e of this block: tiled stage-varying data interleaves 32 stages element-major;
  // halo tiles interleave tw slots and hold the stage up to three times (its own slot and the
  // halo slots of the neighbouring tiles); everything else is a plain block.
  T *bases[3];
  int nb = 1, es;
  if (a.L.tiled == 2) {
    const int tw = a.L.tw[j];
    int t, sl, tt[2], ss[2];
    halo_slot(tw, kb, t, sl);
    es = tw;
    bases[0] = blk + a.L.blk[j] + (int64_t)t * W + sl;
    const int m = halo_copies(tw, N, kb, tt, ss);
    for (int q = 0; q < m; ++q) bases[1 + q] = blk + a.L.blk[j] + (int64_t)tt[q] * W + ss[q];
    nb = 1 + m;
  } else if (lay == 1 && !lti) {
    bases[0] = blk + a.L.blk[j] + (int64_t)(kb >> 5) * 32 * W + (kb & 31);
    es = 32;
  } else {
    bases[0] = blk + a.L.blk[j] + (int64_t)kb * W;
    es = 1;
  }
  auto put = [&](int e, double v) {
    for (int q = 0; q < nb; ++q) bases[q][(int64_t)e * es] = (T)v;
  };
  // Symmetric matrices: packed lower row-major (one-thread-per-stage kernels) or wrapped
  // diagonals, row d holding S[c][(c + d) mod m] (lane-group kernels); H of the blocked layout
  // as wrapped 4 x 4 block diagonals (slot w is element (a, b) of block (d, I), see
  // bl_sym_index).
  auto put_sym_blocks = [&](int o, int m, const double *Xs, int ldx) {
    const int nbm = bl_nb(m);
    for (int w = lane; w < bl_sym_words(m); w += 32) {
      int d, I, a4, b;
      if (!bl_sym_slot(nbm, w, d, I, a4, b)) {  // padding of the diagonal-block region
        put(o + w, 0.0);
        continue;
      }
      const int r = 4 * I + a4, c = 4 * ((I + d) % nbm) + b;
      put(o + w, (r < m && c < m) ? Xs[r * ldx + c] : 0.0);
    }
  };
  auto put_sym = [&](int o, int m, const double *Xs, int ldx) {
    if (packed) {
      for (int i = 0; i < m; ++i)
        for (int c = lane; c <= i; c += 32) put(o + i * (i + 1) / 2 + c, Xs[i * ldx + c]);
    } else {
      const int rows = wrapped_rows(m);
      for (int d = 0; d < rows; ++d)
        for (int c = lane; c < m; c += 32) put(o + d * m + c, Xs[c * ldx + (c + d) % m]);
    }
  };
  if (blocked) put_sym_blocks(oH, n, X, ld);
  else put_sym(oH, n, X, ld);
  __syncwarp();

  // Own-stage G_k, e_k and M_k = (B_k^T B_k + I + Wdu/rho)^{-1}.
  const double *Ak = A + (size_t)kS * nx * nx, *Bk = B + (size_t)kS * nx * nu;
  for (int w = lane; w < nx * n; w += 32) {
    int r = w / n, c = w - r * n;
    double g = c < nx ? Ak[r * nx + c] : Bk[r * nu + (c - nx)];
    G[w] = g;
    put(r * ldg + c, g);
  }
  for (int w = lane; w < nx * (ldg - n); w += 32) {  // row padding
    const int r = w / (ldg - n);
    put(r * ldg + n + (w - r * (ldg - n)), 0.0);
  }
  for (int r = lane; r < nx; r += 32) put(oE + r, e ? e[(size_t)kS * nx + r] : 0.0);
  if (blocked)
    for (int r = nx + lane; r < bl_pad4(nx); r += 32) put(oE + r, 0.0);
  __syncwarp();
  const double *rdu = a.rdu ? a.rdu + a.L.off_n[j] + nx : nullptr;
  for (int t = lane; t < nu * (nu + 1) / 2; t += 32) {
    int i, c;
    tri_index(t, i, c);
    double s = 0.0;
    for (int r = 0; r < nx; ++r) s += G[r * n + nx + i] * G[r * n + nx + c];
    if (i == c) s += 1.0 + (rdu ? rdu[i] / rho : 0.0);
    S[i * nu + c] = s;
  }
  __syncwarp();
  sweep_inverse(S, X, nu, nu, lane, a.err + j);
  put_sym(oM, nu, X, nu);
  if (!packed) {  // padding of a plain or blocked block
    const int end = oM + wrapped_size(nu);
    for (int w = end + lane; w < W; w += 32) put(w, 0.0);
  }
}

}  // namespace

int factorise_smem_words(int max_nx, int max_n) { return max_nx * max_n + 2 * max_n * max_n; }

cudaError_t launch_factorise(const Layout &L, const double *A, const double *B, const double *e,
                             const double *qd, const double *rdu, double rho, const int *binst,
                             const int64_t *bbase, int64_t nblocks, int max_nx, int max_n,
                             int precision, void *blk, int *err, cudaStream_t stream) {
  FactArgs a;
  a.L = L; a.A = A; a.B = B; a.e = e; a.qd = qd; a.rdu = rdu; a.rho = rho;
  a.binst = binst; a.bbase = bbase; a.nblocks = nblocks; a.err = err;
  a.words_per_warp = factorise_smem_words(max_nx, max_n);
  const size_t per_warp = (size_t)a.words_per_warp * sizeof(double);
  int wpc = (int)((96 * 1024) / per_warp);
  if (wpc < 1) wpc = 1;
  if (wpc > 8) wpc = 8;
  const size_t smem = per_warp * wpc;
  const int64_t grid = (nblocks + wpc - 1) / wpc;
  cudaError_t rc = cudaMemsetAsync(err, 0, sizeof(int) * (size_t)L.batch, stream);
  if (rc != cudaSuccess) return rc;
  if (grid == 0) return cudaSuccess;
  if (precision == 0) {
    rc = cudaFuncSetAttribute(factorise_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
    if (rc != cudaSuccess) return rc;
    factorise_kernel<float><<<(unsigned)grid, 32 * wpc, smem, stream>>>(a, (float *)blk);
  } else {
    rc = cudaFuncSetAttribute(factorise_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
    if (rc != cudaSuccess) return rc;
    factorise_kernel<double><<<(unsigned)grid, 32 * wpc, smem, stream>>>(a, (double *)blk);
  }
  return cudaGetLastError();
}

}  // namespace pimpc

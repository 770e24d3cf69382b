// admm.cu -- the piMPC iteration (Algorithm 1) on a batch of instances, one CTA per instance.
//
// One launch solves the whole batch: each CTA takes instances from a work queue ordered by
// decreasing cost (N n^2) and runs Algorithm 1 on it until c^{i+1} <= eps or K_max iterations.
// Every iteration is one sweep over the horizon in chunks of S stages. A chunk's stage blocks
// (G_k = [A_k | B_k], e_k, packed H_k and M_k) are staged in shared memory, with H_k and M_k
// expanded to full symmetric matrices and odd row strides so that row and column accesses are
// free of bank conflicts; the next stage's block is loaded too because step 1 of stage k uses
// Abar_{k+1}. Each stage is handled by a group of g lanes (g = 8, 16 or 32 >= n; lane = vector
// component, two components per lane when n > 32).
//
// Per chunk:  load -> [phase 1: step 1 of Algorithm 1: du_k = M_k (B_k^T w_x + w_u),
//             w = vhat_k - betahat_k; h_k = qbar_k + rho (zhat_k - thetahat_k +
//             Abar_{k+1}^T (zhat_{k+1} - vhat_{k+1} - ebar_{k+1} + lambdahat_{k+1}));
//             xbar_{k+1} = H_k h_k]  -> barrier ->
//             [phase 2: steps 2-3 with xbar_k from the previous stage (or xbar_0): gamma_k,
//             z_{k+1} = Proj((2 (xbar_{k+1} + thetahat + Abar xbar_k + ebar - lambdahat) + gamma)/3),
//             v_k = (z + gamma)/2, the three dual updates, and the step-4 terms of c]
// The hats of Algorithm 1 are never stored: with the momentum factor f_i = (alpha_i - 1) /
// alpha_{i+1} (0 after a restart), hat = cur + f (cur - prev) is formed when cur and prev are
// read; the new iterate overwrites prev, and the roles of the two buffers swap. After the sweep
// the CTA reduces c (warp shuffles, then shared memory), applies the stop test (step 5) and the
// momentum / restart rule (steps 6-7). Every loop is bounded by K_max: nothing waits on another
// CTA.
#include <math.h>

#include "launch.h"

namespace pimpc {

namespace {

constexpr int kNone = 0xFFFF;

template <typename T>
struct AdmmArgs {
  Layout L;
  const T *blk;
  T *it[2];
  int *cur;
  const T *qd, *ref;
  int ref_per_stage;
  const T *lo, *hi, *xb0;
  double rho, eps, eta;
  int max_iters, accel;
  const unsigned char *mask;
  int mask_len;
  const int *order;
  int *counter;
  InstState *st;
  double *u_out, *x_out;
  int warm;
};

// Shared-memory plan of one instance (units: elements of T, then ints for the load map).
struct Plan {
  int n, g, S, ldg, ldh, ldm;
  int oG, oE, oH, oM, SW;   // slot offsets and slot stride
  int nslots;
  int oSlots, oScr, oX, oRed, tWords;  // T-array offsets
  int mapInts;
};

__host__ __device__ inline Plan make_plan(int nx, int nu, int lti, int threads) {
  Plan p;
  p.n = nx + nu;
  p.g = p.n <= 8 ? 8 : (p.n <= 16 ? 16 : 32);
  p.S = threads / p.g;
  p.ldg = p.n | 1;
  p.ldh = p.n | 1;
  p.ldm = nu | 1;
  p.oG = 0;
  p.oE = nx * p.ldg;
  p.oH = p.oE + nx;
  p.oM = p.oH + p.n * p.ldh;
  p.SW = p.oM + nu * p.ldm;
  p.SW += (p.SW & 1);
  p.nslots = lti ? 2 : p.S + 1;
  p.oSlots = 0;
  p.oScr = p.nslots * p.SW;
  const int nv = (p.n + 1) & ~1;
  p.oX = p.oScr + p.S * 4 * nv;
  p.oRed = p.oX + (p.S + 1) * nv;
  p.tWords = p.oRed + 64;
  p.mapInts = block_words(nx, nu);
  return p;
}

template <typename T>
__host__ __device__ inline size_t plan_bytes(const Plan &p) {
  return (size_t)p.tWords * sizeof(T) + (size_t)p.mapInts * sizeof(int) + 64;
}

__device__ inline int tri_row(int w) {
  // largest i with i (i + 1) / 2 <= w
  int i = (int)((sqrtf(8.0f * (float)w + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= w) ++i;
  while (i * (i + 1) / 2 > w) --i;
  return i;
}

template <typename T>
__device__ inline T clampv(T x, T lo, T hi) {
  return x < lo ? lo : (x > hi ? hi : x);
}

template <typename T>
__global__ void __launch_bounds__(256) admm_kernel(AdmmArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  __shared__ int sInst;
  __shared__ double sCoef;
  __shared__ int sStop;

  const int tid = threadIdx.x;
  const int nthreads = blockDim.x;
  const int lti = a.L.lti;

  for (;;) {
    __syncthreads();
    if (tid == 0) sInst = atomicAdd(a.counter, 1);
    __syncthreads();
    const int q = sInst;
    if (q >= a.L.batch) break;
    const int j = a.order[q];
    const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j];
    const Plan P = make_plan(nx, nu, lti, nthreads);
    const int n = P.n, g = P.g, S = P.S;
    int *map = reinterpret_cast<int *>(sm + P.tWords);
    T *slots = sm + P.oSlots;
    T *X = sm + P.oX;
    T *red = sm + P.oRed;
    const int nv = (n + 1) & ~1;

    const int W = a.L.W[j];
    const T *blk = a.blk + a.L.blk[j];
    const int64_t ibase = 5 * a.L.Nn[j];
    const T *qd = a.qd + a.L.off_n[j];
    const T *ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
    const int refstride = a.ref_per_stage ? n : 0;
    const T *lo = a.lo + a.L.off_n[j];
    const T *hi = a.hi + a.L.off_n[j];
    const T *xb0 = a.xb0 + a.L.off_n[j];
    const T rho = (T)a.rho;
    int cur = a.cur[j];

    // Load map of a stage block into the expanded slot layout.
    for (int w = tid; w < W; w += nthreads) {
      int d1 = kNone, d2 = kNone;
      const int nG = nx * n, nE = nx, nH = n * (n + 1) / 2, nM = nu * (nu + 1) / 2;
      if (w < nG) {
        int r = w / n, c = w - r * n;
        d1 = P.oG + r * P.ldg + c;
      } else if (w < nG + nE) {
        d1 = P.oE + (w - nG);
      } else if (w < nG + nE + nH) {
        int t = w - nG - nE;
        int i = tri_row(t), c = t - i * (i + 1) / 2;
        d1 = P.oH + i * P.ldh + c;
        if (c != i) d2 = P.oH + c * P.ldh + i;
      } else if (w < nG + nE + nH + nM) {
        int t = w - nG - nE - nH;
        int i = tri_row(t), c = t - i * (i + 1) / 2;
        d1 = P.oM + i * P.ldm + c;
        if (c != i) d2 = P.oM + c * P.ldm + i;
      }
      map[w] = d1 | (d2 << 16);
    }
    // Starting iterates: cold start zeroes the current buffer; mode 2 shifts it one stage.
    if (a.warm == 0) {
      T *dst = a.it[cur] + ibase;
      for (int64_t t = tid; t < (int64_t)5 * N * n; t += nthreads) dst[t] = (T)0;
    } else if (a.warm == 2) {
      const T *src = a.it[cur] + ibase;
      T *dst = a.it[cur ^ 1] + ibase;
      for (int64_t t = tid; t < (int64_t)5 * N * n; t += nthreads) {
        int k = (int)(t / (5 * n));
        int r = (int)(t - (int64_t)k * 5 * n);
        int ks = k + 1 < N ? k + 1 : N - 1;
        dst[t] = src[(int64_t)ks * 5 * n + r];
      }
      cur ^= 1;
    }
    __syncthreads();
    // LTI: both stage blocks (H_k and H_{N-1}) stay in shared memory for the whole solve.
    if (lti) {
      for (int t = tid; t < 2 * W; t += nthreads) {
        int s = t / W, w = t - s * W;
        int m = map[w];
        T v = blk[t];
        int d1 = m & 0xFFFF, d2 = (m >> 16) & 0xFFFF;
        if (d1 != kNone) slots[s * P.SW + d1] = v;
        if (d2 != kNone) slots[s * P.SW + d2] = v;
      }
    }

    const int grp = tid / g;
    const int l = tid - grp * g;
    T *scr = sm + P.oScr + grp * 4 * nv;
    T *sW = scr, *sY = scr + nv, *sH = scr + 2 * nv, *sDU = scr + 3 * nv;
    const int ncl = (g == 32 && n > 32) ? 2 : 1;

    double alpha = 1.0, c_prev = 1.0, coef = 0.0, c_last = 0.0;
    int status = kMaxIter, iters = 0, nmom = 0;
    for (int it = 0; it < a.max_iters; ++it) {
      const T f = (T)coef;
      nmom += coef != 0.0;
      const bool use_prev = coef != 0.0;
      const T *Bc = a.it[cur] + ibase;
      const T *Bp = a.it[cur ^ 1] + ibase;
      T *Bn = a.it[cur ^ 1] + ibase;
      T cacc = (T)0;
      for (int k0 = 0; k0 < N; k0 += S) {
        const int cnt = min(S, N - k0);
        // ---- load the chunk's stage blocks (plus the next stage's) ----
        if (!lti) {
          const int nst = cnt + (k0 + cnt < N ? 1 : 0);
          const T *src = blk + (int64_t)k0 * W;
          for (int t = tid; t < nst * W; t += nthreads) {
            int s = t / W, w = t - s * W;
            int m = map[w];
            T v = src[t];
            int d1 = m & 0xFFFF, d2 = (m >> 16) & 0xFFFF;
            if (d1 != kNone) slots[s * P.SW + d1] = v;
            if (d2 != kNone) slots[s * P.SW + d2] = v;
          }
        }
        if (k0 == 0)
          for (int c = tid; c < n; c += nthreads) X[c] = xb0[c];
        __syncthreads();

        // ---- phase 1: step 1 (du_k and xbar_{k+1}) ----
        T zh[2], vh[2], thh[2], beh[2], lah[2];
        const int k = k0 + grp;
        const bool active = grp < cnt;
        const T *Sk = slots + (lti ? ((k < N - 1) ? 0 : P.SW) : grp * P.SW);
        const T *Gk = lti ? slots : slots + grp * P.SW;         // G_k, e_k, M_k
        const T *Gk1 = lti ? slots : slots + (grp + 1) * P.SW;  // G_{k+1}, e_{k+1}
        if (active) {
          const T *c0 = Bc + (int64_t)k * 5 * n;
          const T *p0 = Bp + (int64_t)k * 5 * n;
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T cz = c0[c], cv = c0[n + c], ct = c0[2 * n + c], cb = c0[3 * n + c], cl = c0[4 * n + c];
              if (use_prev) {
                cz += f * (cz - p0[c]);
                cv += f * (cv - p0[n + c]);
                ct += f * (ct - p0[2 * n + c]);
                cb += f * (cb - p0[3 * n + c]);
                cl += f * (cl - p0[4 * n + c]);
              }
              zh[qq] = cz; vh[qq] = cv; thh[qq] = ct; beh[qq] = cb; lah[qq] = cl;
              sW[c] = cv - cb;
              T y = (T)0;
              if (k + 1 < N) {
                const T *c1 = c0 + 5 * n, *p1 = p0 + 5 * n;
                T nz = c1[c], nvv = c1[n + c], nl = c1[4 * n + c];
                if (use_prev) {
                  nz += f * (nz - p1[c]);
                  nvv += f * (nvv - p1[n + c]);
                  nl += f * (nl - p1[4 * n + c]);
                }
                y = nz - nvv + nl - (c < nx ? Gk1[P.oE + c] : (T)0);
              }
              sY[c] = y;
            }
          }
        }
        __syncwarp();
        if (active && l < nu) {
          // t = B_k^T w_x + w_u
          const int c = l;
          T t = sW[nx + c];
          for (int r = 0; r < nx; ++r) t += Gk[P.oG + r * P.ldg + nx + c] * sW[r];
          sH[c] = t;
        }
        __syncwarp();
        if (active && l < nu) {
          // du_k = M_k t
          const int c = l;
          T d = (T)0;
          for (int cc = 0; cc < nu; ++cc) d += Gk[P.oM + cc * P.ldm + c] * sH[cc];
          sDU[c] = d;
        }
        __syncwarp();
        if (active) {
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T acc = (T)0;
              if (k + 1 < N) {
                // Abar_{k+1}^T y = G_{k+1}^T y_x + (0, y_u)
                for (int r = 0; r < nx; ++r) acc += Gk1[P.oG + r * P.ldg + c] * sY[r];
                if (c >= nx) acc += sY[c];
              }
              const T rf = ref ? ref[(int64_t)k * refstride + c] : (T)0;
              sH[c] = qd[c] * rf + rho * (zh[qq] - thh[qq] + acc);
            }
          }
        }
        __syncwarp();
        if (active) {
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T acc = (T)0;
              for (int cc = 0; cc < n; ++cc) acc += Sk[P.oH + cc * P.ldh + c] * sH[cc];
              X[(grp + 1) * nv + c] = acc;
            }
          }
        }
        __syncthreads();

        // ---- phase 2: steps 2-4 ----
        if (active) {
          const T *xk = X + grp * nv;          // xbar_k
          const T *xk1 = X + (grp + 1) * nv;   // xbar_{k+1}
          T *o = Bn + (int64_t)k * 5 * n;
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T ax, bd, ee;
              if (c < nx) {
                T s1 = (T)0, s2 = (T)0;
                const T *row = Gk + P.oG + c * P.ldg;
                for (int cc = 0; cc < n; ++cc) s1 += row[cc] * xk[cc];
                for (int cc = 0; cc < nu; ++cc) s2 += row[nx + cc] * sDU[cc];
                ax = s1; bd = s2; ee = Gk[P.oE + c];
              } else {
                ax = xk[c]; bd = sDU[c - nx]; ee = (T)0;
              }
              const T xn = xk1[c];
              const T gam = bd + beh[qq] - ax - ee + lah[qq];
              const T w = ((T)2 * (xn + thh[qq] + ax + ee - lah[qq]) + gam) / (T)3;
              const T z = clampv(w, lo[c], hi[c]);
              const T v = (T)0.5 * (z + gam);
              const T th = thh[qq] + xn - z;
              const T be = beh[qq] + bd - v;
              const T la = lah[qq] + z - ax - v - ee;
              const T d1 = th - thh[qq], d2 = be - beh[qq], d3 = la - lah[qq];
              const T d4 = z - zh[qq], d5 = v - vh[qq], d6 = d4 - d5;
              cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
              o[c] = z; o[n + c] = v; o[2 * n + c] = th; o[3 * n + c] = be; o[4 * n + c] = la;
            }
          }
        }
        __syncthreads();
        // xbar at the end of this chunk becomes xbar_k of the next chunk's first stage
        for (int c = tid; c < n; c += nthreads) X[c] = X[cnt * nv + c];
      }
      // ---- step 4: reduce c; steps 5-7 ----
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if ((tid & 31) == 0) red[tid >> 5] = cacc;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (nthreads >> 5); ++w) s += (double)red[w];
        const double c = (double)rho * s;
        int stop = 0;
        if (!isfinite(c)) {
          status = kNonFinite; stop = 1;
        } else if (c <= a.eps) {
          status = kConverged; stop = 1;
        } else {
          int take = 0;
          if (a.accel) {
            if (a.mask && it < a.mask_len) take = a.mask[(int64_t)j * a.mask_len + it] != 0;
            else take = c <= a.eta * c_prev;
          }
          if (take) {
            const double an = 0.5 + 0.5 * sqrt(1.0 + 4.0 * alpha * alpha);
            coef = (alpha - 1.0) / an;
            alpha = an;
          } else {
            alpha = 1.0;
            coef = 0.0;
          }
          c_prev = c;
        }
        c_last = c;
        sCoef = coef;
        sStop = stop;
      }
      __syncthreads();
      coef = sCoef;
      cur ^= 1;
      iters = it + 1;
      if (sStop) break;
    }
    // Outputs: u_k and x_{k+1} from z_{k+1} of the latest iterate.
    const T *Bf = a.it[cur] + ibase;
    if (a.x_out || a.u_out) {
      for (int64_t t = tid; t < (int64_t)N * n; t += nthreads) {
        int k = (int)(t / n), c = (int)(t - (int64_t)k * n);
        double zval = (double)Bf[(int64_t)k * 5 * n + c];
        if (c < nx) {
          if (a.x_out) a.x_out[a.L.Nnx[j] + (int64_t)k * nx + c] = zval;
        } else if (a.u_out) {
          a.u_out[a.L.Nnu[j] + (int64_t)k * nu + (c - nx)] = zval;
        }
      }
    }
    if (tid == 0) {
      a.cur[j] = cur;
      a.st[j].iters = iters;
      a.st[j].status = status;
      a.st[j].c = c_last;
      a.st[j].momentum = nmom;
    }
  }
}

}  // namespace

int admm_threads(int precision) { return precision == 0 ? 256 : 128; }

size_t admm_smem_bytes(int nx, int nu, int lti, int threads, int precision) {
  Plan p = make_plan(nx, nu, lti, threads);
  return precision == 0 ? plan_bytes<float>(p) : plan_bytes<double>(p);
}

cudaError_t admm_configure(int precision, size_t smem, int *blocks_per_sm) {
  cudaError_t rc;
  const int threads = admm_threads(precision);
  if (precision == 0) {
    rc = cudaFuncSetAttribute(admm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, admm_kernel<float>, threads, smem);
  } else {
    rc = cudaFuncSetAttribute(admm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, admm_kernel<double>, threads, smem);
  }
  return rc;
}

template <typename T>
static AdmmArgs<T> make_args(const AdmmLaunch &s) {
  AdmmArgs<T> a;
  a.L = s.L;
  a.blk = (const T *)s.blk;
  a.it[0] = (T *)s.it0;
  a.it[1] = (T *)s.it1;
  a.cur = s.cur;
  a.qd = (const T *)s.qd;
  a.ref = (const T *)s.ref;
  a.ref_per_stage = s.ref_per_stage;
  a.lo = (const T *)s.lo;
  a.hi = (const T *)s.hi;
  a.xb0 = (const T *)s.xb0;
  a.rho = s.rho; a.eps = s.eps; a.eta = s.eta;
  a.max_iters = s.max_iters; a.accel = s.accel;
  a.mask = s.mask; a.mask_len = s.mask_len;
  a.order = s.order; a.counter = s.counter; a.st = s.st;
  a.u_out = s.u_out; a.x_out = s.x_out; a.warm = s.warm;
  return a;
}

cudaError_t launch_admm(const AdmmLaunch &s, int precision, int grid, size_t smem,
                        cudaStream_t stream) {
  const int threads = admm_threads(precision);
  if (precision == 0)
    admm_kernel<float><<<grid, threads, smem, stream>>>(make_args<float>(s));
  else
    admm_kernel<double><<<grid, threads, smem, stream>>>(make_args<double>(s));
  return cudaGetLastError();
}

}  // namespace pimpc

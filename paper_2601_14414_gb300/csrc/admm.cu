// admm.cu -- Algorithm 1 with a group of lanes per stage on plain stage blocks, one component per
// lane (schedule family 0, the default for FP64 iterations; FP32 iterations default to the
// blocked lane groups of admm_blk.cu).
//
// Work decomposition. The stages of every instance are cut into items of consecutive stages
// (item = instance j, stages [a, b)). One cooperative launch runs all iterations of all
// instances in lock-step: in iteration i every CTA pulls items from a queue and runs the
// iteration on their stages; a grid barrier separates iterations. Because Algorithm 1 is
// parallel in the horizon (every update of stage k reads only stages k-1, k and k+1), an item
// needs one stage of halo on each side: the block and hats of stage a-1 to recompute
// xbar_a = H_{a-1} h_{a-1}, and G_b, e_b and the hats of stage b for h_{b-1}. Each item stores
// its share of c^{i+1}; after the barrier one thread per instance sums the shares and applies the
// stop test (step 5) and the momentum / restart rule (steps 6-7) for that instance. Stopped
// instances leave the queue (stream compaction after the barrier), so the
// remaining instances keep every SM busy and an instance that needs many iterations is spread
// over many CTAs instead of running alone.
//
// Data movement. Stage blocks (G_k = [A_k | B_k] row-major, e_k, H_k and M_k stored diagonal by
// diagonal) and the iterates of a sub-chunk of S stages (plus the next stage) arrive in shared
// memory by cp.async.bulk copies completing on an mbarrier; with one buffer (the default) the
// copies of the next sub-chunk are issued after the current one is computed and the other CTAs
// resident on the SM hide the latency, with two buffers they overlap the compute. Every wait is
// bounded; a timeout raises an error flag that ends the launch (no instance is marked
// converged).
//
// Iterates. Three buffers rotate: iteration i reads cur = buf[(base + i) % 3] and, when the
// momentum factor f_i = (alpha_i - 1) / alpha_{i+1} is nonzero, prev = buf[(base + i - 1) % 3];
// the hats of Algorithm 1 are formed on the fly (hat = cur + f (cur - prev)) and the new
// iterate goes to the third buffer, so neighbouring items of the same instance never read
// what another CTA writes in the same iteration.
//
// Compute. A group of g lanes (8, 16 or 32 >= n; two components per lane when n > 32) handles one
// stage. Phase 1 (step 1): du_k = M_k (B_k^T w_x + w_u), w = vhat_k - betahat_k;
// h_k = qbar_k + rho (zhat_k - thetahat_k + Abar_{k+1}^T (zhat_{k+1} - vhat_{k+1} - ebar_{k+1} +
// lambdahat_{k+1})); xbar_{k+1} = H_k h_k. Phase 2 (steps 2-4) with xbar_k of the previous stage:
// gamma_k, z_{k+1} = Proj((2 (xbar_{k+1} + thetahat + Abar xbar_k + ebar - lambdahat) + gamma)/3),
// v_k = (z + gamma) / 2, the three dual updates and the six squared norms of c.
#include <math.h>

#include <algorithm>

#include "bulk.cuh"
#include "usets.cuh"
#include "lockstep.cuh"
#include "products.cuh"

namespace pimpc {

__global__ void set_control_kernel(Ctl *c, int nitems, int batch, int bar_limit) {
  c->bar_limit = bar_limit;
  c->nlist[0] = nitems;
  c->nlist[1] = 0;
  c->active = batch;
}

namespace {

using ls::kWaitLimit;
using namespace bulk;

template <typename T>
using Args = ls::Args<T>;

__host__ __device__ inline int group_size(int n) { return n <= 8 ? 8 : (n <= 16 ? 16 : 32); }
__host__ __device__ inline int iter_stride(int n, int tsize) {
  const int q = 16 / tsize;  // 16-byte granules
  return (5 * n + q - 1) / q * q;
}

// Shared-memory layout of a launch (sized by the largest instance of the batch), in elements.
struct Smem {
  int nbuf, rawB, capB, rawI, capI, haloB, haloI, scr, X, total;
};

// nbuf = 2: the copies of sub-chunk s+1 overlap the compute of sub-chunk s inside the CTA;
// nbuf = 1: one buffer, and the overlap comes from the other CTAs resident on the SM.
__host__ __device__ inline Smem smem_layout(int capB, int capI, int haloB, int haloI, int S_max,
                                            int nv_max, int tsize, int nbuf) {
  const int q = 16 / tsize;
  auto up = [q](int v) { return (v + q - 1) / q * q; };
  Smem s;
  s.nbuf = nbuf;
  s.capB = up(capB);
  s.capI = up(capI);
  s.rawB = 0;
  s.rawI = s.rawB + nbuf * s.capB;
  s.haloB = s.rawI + 2 * nbuf * s.capI;  // per buffer: cur, then prev
  s.haloI = s.haloB + up(haloB);
  s.scr = s.haloI + up(haloI);
  s.X = s.scr + up(S_max);         // S_max here carries max_j S_j * 4 * nv_j (group scratch)
  s.total = s.X + up(nv_max);       // nv_max here carries max_j 2 (S_j + 1) nv_j (xbar rows)
  return s;
}

template <typename T>
__device__ inline T clampv(T x, T lo, T hi) {
  return x < lo ? lo : (x > hi ? hi : x);
}


// ---------------------------------------------------------------------------------------------
// The persistent kernel.
// ---------------------------------------------------------------------------------------------
// kSets: compiled with the projection onto non-box input sets (see the blocked kernel).
template <typename T, bool kSets>
__global__ void __launch_bounds__(256, 3) admm_kernel(Args<T> a, Smem lay) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int sItem, sOk, sArr;
  __shared__ double sRed[8];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x;
  const int nthreads = blockDim.x;
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;
  const int lti = a.L.lti;

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par[2] = {0u, 0u};
  bool pend[2] = {false, false};

  int cl = 0;
  for (int it = 0; it < a.max_iters; ++it) {
    const int nact = *(volatile int *)&ctl->nlist[cl];
    bool ok = true;
    for (;;) {
      if (tid == 0) sItem = atomicAdd(&ctl->queue[it & 1], 1);
      __syncthreads();
      const int q = sItem;
      __syncthreads();
      if (q >= nact) break;
      const int item = a.list[cl][q];
      if (item < 0) continue;  // an entry of an instance that has stopped
      const int j = a.item_inst[item];
      if (*(volatile int *)&a.stop[j]) continue;
      const int ka = a.item_a[item], kb = a.item_b[item];
      const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
      const int g = group_size(n), S = nthreads / g, nv = (n + 3) & ~3;
      const int n5p = iter_stride(n, (int)sizeof(T));
      const int W = a.L.W[j];
      const int ldg = odd_ld(n);
      const int bse = a.base[j];
      const int64_t ib = a.L.Ni[j];
      const T *Ic = a.it[(bse + it) % 3] + ib;
      const T *Ip = a.it[(bse + it + 2) % 3] + ib;
      T *In = a.it[(bse + it + 1) % 3] + ib;
      const T *blk = a.blk + a.L.blk[j];
      const double coefd = *(volatile double *)&a.coef[j];
      const T f = (T)coefd;
      const bool use_prev = coefd != 0.0;
      const T rho = (T)a.rho;
      const T *qd = a.qd + a.L.off_n[j];
      const T *ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
      const int refstride = a.ref_per_stage ? n : 0;
      const T *lo = a.lo + a.L.off_n[j], *hi = a.hi + a.L.off_n[j];
      const int ukind = kSets && a.uset_kind ? a.uset_kind[j] : uset::kUsetBox;  // input set U
      const T ur = kSets && a.uset_kind ? a.uset_r[j] : (T)0;
      const T *ua = kSets && a.uset_a ? a.uset_a + a.L.off_n[j] : nullptr;
      const int grp = tid / g, l = tid - grp * g;
      const unsigned gmask = g == 32 ? 0xffffffffu : (((1u << g) - 1u) << ((tid & 31) & ~(g - 1)));
      const int ncl = (g == 32 && n > 32) ? 2 : 1;
      T *scr = sm + lay.scr + grp * 4 * nv;
      T *sW = scr, *sY = scr + nv, *sH = scr + 2 * nv, *sDU = scr + 3 * nv;
      T *haloB = sm + lay.haloB, *haloI = sm + lay.haloI;
      const T *ltiB = haloB;  // LTI: block 0 (H_k, k < N-1) then block 1 (H_{N-1})
      const int oE = nx * ldg, oH = oE + nx, oM = oH + wrapped_size(n);
      T cacc = (T)0;

      // Copies of the sub-chunk that starts at stage k0 into buffer b (thread 0 issues).
      auto issue = [&](int k0, int b, bool first) {
        const int cnt = min(S, kb - k0);
        const int la = (k0 + cnt < N) ? 1 : 0;  // the next stage: its G and e only
        const int ns = cnt + la;
        const bool halo = first && ka > 0;
        const uint32_t it_bytes = (uint32_t)(ns * n5p * sizeof(T));
        const uint32_t blk_bytes = (uint32_t)((cnt * W + la * ((oE + nx + 3) & ~3)) * sizeof(T));
        uint32_t bytes = it_bytes * (use_prev ? 2u : 1u);
        if (!lti) bytes += blk_bytes;
        if (halo) {
          bytes += (uint32_t)(n5p * sizeof(T)) * (use_prev ? 2u : 1u);
          if (!lti) bytes += (uint32_t)(W * sizeof(T));
        }
        if (lti && first) bytes += (uint32_t)(2 * W * sizeof(T));
        // The iterates the copies read were written through the generic proxy by other CTAs
        // before the grid barrier: one proxy fence after that barrier, i.e. at the item's first
        // copy, orders them before every later copy of the item. (The shared-memory buffer the
        // copies overwrite was only read, and those reads precede the CTA barrier.)
        if (first) fence_proxy_async();
        mbar_expect_tx(&mbar[b], bytes);
        T *rB = sm + lay.rawB + b * lay.capB;
        T *rI = sm + lay.rawI + b * 2 * lay.capI;
        if (!lti) bulk_load(rB, blk + (int64_t)k0 * W, blk_bytes, &mbar[b]);
        bulk_load(rI, Ic + (int64_t)k0 * n5p, it_bytes, &mbar[b]);
        if (use_prev) bulk_load(rI + lay.capI, Ip + (int64_t)k0 * n5p, it_bytes, &mbar[b]);
        if (halo) {
          if (!lti) bulk_load(haloB, blk + (int64_t)(ka - 1) * W, (uint32_t)(W * sizeof(T)), &mbar[b]);
          bulk_load(haloI, Ic + (int64_t)(ka - 1) * n5p, (uint32_t)(n5p * sizeof(T)), &mbar[b]);
          if (use_prev)
            bulk_load(haloI + n5p, Ip + (int64_t)(ka - 1) * n5p, (uint32_t)(n5p * sizeof(T)), &mbar[b]);
        }
        if (lti && first) bulk_load(haloB, blk, (uint32_t)(2 * W * sizeof(T)), &mbar[b]);
      };

      const int nsub = (kb - ka + S - 1) / S;
      if (tid == 0) issue(ka, 0, true);
      pend[0] = true;
      int b = 0;
      for (int sc = 0; sc < nsub; ++sc, b ^= (lay.nbuf - 1)) {
        const int k0 = ka + sc * S;
        const int cnt = min(S, kb - k0);
        if (lay.nbuf == 2 && sc + 1 < nsub) {
          if (tid == 0) issue(k0 + S, b ^ 1, false);
          pend[b ^ 1] = true;
        } else if (lay.nbuf == 1 && sc > 0) {
          if (tid == 0) issue(k0, 0, false);  // the single buffer is free after the last barrier
          pend[0] = true;
        }
        // One thread waits on the copies; the others wait at the barrier without issuing.
        if (tid == 0) sArr = mbar_wait(&mbar[b], par[b], ctl) ? 1 : 0;
        __syncthreads();
        const bool arrived = sArr != 0;
        if (arrived) {
          par[b] ^= 1u;
          pend[b] = false;
        } else {
          ok = false;  // the copy may still be in flight: it stays pending for the exit wait
        }
        const T *rB = sm + lay.rawB + b * lay.capB;
        const T *rIc = sm + lay.rawI + b * 2 * lay.capI;
        const T *rIp = rIc + lay.capI;
        // xbar rows: Xc for this sub-chunk; the last stage also seeds row 0 of the next one
        T *Xc = sm + lay.X + (sc & 1) * (S + 1) * nv;
        T *Xn = sm + lay.X + ((sc & 1) ^ 1) * (S + 1) * nv;

        // ---- phase 1: step 1 ----
        T zh[2], vh[2], thh[2], beh[2], lah[2];
        const int k = k0 + grp;
        const bool active = arrived && grp < cnt;
        const T *Hk = lti ? (ltiB + ((k < N - 1) ? 0 : W)) : rB + grp * W;  // block holding H_k
        const T *Gk = lti ? ltiB : rB + grp * W;                           // G_k, e_k, M_k
        const T *Gk1 = lti ? ltiB : rB + (grp + 1) * W;                    // G_{k+1}, e_{k+1}
        const T *hc = rIc + grp * n5p, *hp = rIp + grp * n5p;
        if (active) {
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T cz = hc[c], cv = hc[n + c], ct = hc[2 * n + c], cb = hc[3 * n + c], cm = hc[4 * n + c];
              if (use_prev) {
                cz += f * (cz - hp[c]);
                cv += f * (cv - hp[n + c]);
                ct += f * (ct - hp[2 * n + c]);
                cb += f * (cb - hp[3 * n + c]);
                cm += f * (cm - hp[4 * n + c]);
              }
              zh[qq] = cz; vh[qq] = cv; thh[qq] = ct; beh[qq] = cb; lah[qq] = cm;
              sW[c] = cv - cb;
              T y = (T)0;
              if (k + 1 < N) {
                const T *nc = hc + n5p, *np = hp + n5p;
                T nz = nc[c], nvv = nc[n + c], nl = nc[4 * n + c];
                if (use_prev) {
                  nz += f * (nz - np[c]);
                  nvv += f * (nvv - np[n + c]);
                  nl += f * (nl - np[4 * n + c]);
                }
                y = nz - nvv + nl - (c < nx ? Gk1[oE + c] : (T)0);
              }
              sY[c] = y;
            }
          }
        }
        __syncwarp();
        if (active && l < nu) sH[l] = sW[nx + l] + dot_col(Gk + nx + l, ldg, sW, nx);  // B_k^T w_x + w_u
        __syncwarp();
        if (active && l < nu) sDU[l] = sym_wrapped(Gk + oM, sH, nu, l);  // du_k = M_k t
        __syncwarp();
        if (active) {
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T acc = (T)0;
              if (k + 1 < N) {  // Abar_{k+1}^T y = G_{k+1}^T y_x + (0, y_u)
                acc = dot_col(Gk1 + c, ldg, sY, nx);
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
              const T xn = sym_wrapped(Hk + oH, sH, n, c);  // xbar_{k+1} = H_k h_k
              Xc[(grp + 1) * nv + c] = xn;
              if (grp + 1 == cnt) Xn[c] = xn;
            }
          }
        }
        // xbar_k of the first stage: xbar_0, or (first sub-chunk of an item that starts at
        // a > 0) H_{a-1} h_{a-1} recomputed from the halo; later sub-chunks got it above.
        if (sc == 0) {
          if (ka == 0) {
            for (int c = tid; c < n; c += nthreads) Xc[c] = a.xb0[a.L.off_n[j] + c];
          } else if (grp == 0 && arrived) {
            __syncwarp(gmask);
            for (int qq = 0; qq < ncl; ++qq) {  // y_a from this group's own hats (stage a)
              const int c = l + 32 * qq;
              if (c < n) sY[c] = zh[qq] - vh[qq] + lah[qq] - (c < nx ? Gk[oE + c] : (T)0);
            }
            __syncwarp(gmask);
            const T *hcm = haloI, *hpm = haloI + n5p;
            const T *Hm = lti ? ltiB : haloB;  // a - 1 < N - 1
            for (int qq = 0; qq < ncl; ++qq) {
              const int c = l + 32 * qq;
              if (c < n) {
                T acc = dot_col(Gk + c, ldg, sY, nx);
                if (c >= nx) acc += sY[c];
                T zm = hcm[c], tm = hcm[2 * n + c];
                if (use_prev) {
                  zm += f * (zm - hpm[c]);
                  tm += f * (tm - hpm[2 * n + c]);
                }
                const T rf = ref ? ref[(int64_t)(ka - 1) * refstride + c] : (T)0;
                sW[c] = qd[c] * rf + rho * (zm - tm + acc);
              }
            }
            __syncwarp(gmask);
            for (int qq = 0; qq < ncl; ++qq) {
              const int c = l + 32 * qq;
              if (c < n) Xc[c] = sym_wrapped(Hm + oH, sW, n, c);
            }
          }
        }
        if (!__syncthreads_and(arrived)) { ok = false; break; }  // uniform across the CTA

        // ---- phase 2: steps 2-4 ----
        {
          const T *xk = Xc + grp * nv;
          const T *xk1 = Xc + (grp + 1) * nv;
          T *o = In + (int64_t)k * n5p;
          T wv[2] = {(T)0, (T)0}, gv[2], axv[2], bdv[2], eev[2], xnv[2], av[2] = {(T)0, (T)0};
          int cv[2] = {-1, -1};
          for (int qq = 0; qq < ncl && active; ++qq) {
            const int c = l + 32 * qq;
            if (c < n) {
              T ax, bd, ee;
              if (c < nx) {
                const T *row = Gk + c * ldg;  // odd stride: the lanes' rows hit distinct banks
                ax = dot_col(row, 1, xk, n);
                bd = dot_col(row + nx, 1, sDU, nu);
                ee = Gk[oE + c];
              } else {
                ax = xk[c]; bd = sDU[c - nx]; ee = (T)0;
              }
              const T xn = xk1[c];
              cv[qq] = c;
              axv[qq] = ax; bdv[qq] = bd; eev[qq] = ee; xnv[qq] = xn;
              gv[qq] = bd + beh[qq] - ax - ee + lah[qq];
              wv[qq] = ((T)2 * (xn + thh[qq] + ax + ee - lah[qq]) + gv[qq]) / (T)3;
              if (ukind == uset::kUsetHalfspace) av[qq] = ua[c];
            }
          }
          // Input part onto a non-box set U (warp-wide; the kind is the same for the CTA's item).
          if (kSets && ukind != uset::kUsetBox)
            uset::project_inputs<T, 2>(ukind, ur, av, wv, cv, nx, n, g,
                                       [](int jj) { return jj & 31; }, [](int jj) { return jj >> 5; });
          for (int qq = 0; qq < ncl && active; ++qq) {
            const int c = cv[qq];
            if (c >= 0) {
              const T ax = axv[qq], bd = bdv[qq], ee = eev[qq], xn = xnv[qq], gam = gv[qq];
              const T z = (c < nx || ukind == uset::kUsetBox) ? clampv(wv[qq], lo[c], hi[c]) : wv[qq];
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
      }
      if (!ok) break;

      // ---- step 4: this item's share of c (steps 5-7 follow in the pass after the barrier) ----
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if ((tid & 31) == 0) sRed[tid >> 5] = (double)cacc;
      __syncthreads();
      if (tid == 0) {
        double part = 0.0;
        for (int w = 0; w < (nthreads >> 5); ++w) part += sRed[w];
        a.cpart[item] = part;  // steps 5-7 run in the pass after the barrier
      }
    }
    if (blockIdx.x == 0 && tid == 0) ctl->queue[(it + 1) & 1] = 0;
    if (!ls::grid_sync(ctl, nblocks, &sOk)) break;
    if (!ls::finish_pass(a, it, cl, nblocks, &sOk)) break;
    if (*(volatile int *)&ctl->active <= 0) break;
    if (!ls::compact(a, cl, nact, &sOk, reinterpret_cast<int *>(sRed))) break;
  }
  // Never leave a bulk copy in flight into shared memory: wait (bounded) for pending phases.
  for (int b = 0; b < 2; ++b)
    if (pend[b]) {
      long long k = 0;
      while (!mbar_try_wait(&mbar[b], par[b]) && ++k < kWaitLimit) {
      }
    }
}

template <typename T>
Smem layout_of(const AdmmLaunch &s) {
  return smem_layout(s.capB, s.capI, s.haloB, s.haloI, s.S_max, s.nv_max, (int)sizeof(T), s.nbuf);
}

template <typename T>
cudaError_t launch_t(const AdmmLaunch &s, cudaStream_t stream) {
  Args<T> a = ls::make_args<T>(s);
  Smem lay = layout_of<T>(s);
  a.capI = lay.capI;
  void *params[] = {&a, &lay};
  return ls::launch_sequence<T>(s, a, s.uset_kind ? (const void *)admm_kernel<T, true> : (const void *)admm_kernel<T, false>, params,
                                (size_t)lay.total * sizeof(T), stream);
}

}  // namespace

int admm_threads(int precision) { return precision == 0 ? 256 : 128; }
int admm_iter_stride(int n, int precision) { return iter_stride(n, precision == 0 ? 4 : 8); }
int admm_group_size(int n) { return group_size(n); }

size_t admm_smem_bytes(const AdmmLaunch &s, int precision) {
  if (precision == 0) return (size_t)layout_of<float>(s).total * 4;
  return (size_t)layout_of<double>(s).total * 8;
}

cudaError_t admm_configure(int precision, size_t smem, int *blocks_per_sm) {
  cudaError_t rc;
  const int threads = admm_threads(precision);
  if (precision == 0) {
    rc = cudaFuncSetAttribute(admm_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, admm_kernel<float, false>, threads, smem);
  } else {
    rc = cudaFuncSetAttribute(admm_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, admm_kernel<double, false>, threads, smem);
  }
  return rc;
}

cudaError_t launch_admm(const AdmmLaunch &s, int precision, cudaStream_t stream) {
  return precision == 0 ? launch_t<float>(s, stream) : launch_t<double>(s, stream);
}

}  // namespace pimpc

// admm_tb.cu -- temporal blocking of the plain iteration (schedule family 7).
//
// Every update of stage k in an iteration of Algorithm 1 (plain form, hats = iterates) reads
// only stages k - 1, k and k + 1: step 1 at stage k reads the iterates of stages k and k + 1,
// step 2 at stage k reads xbar_k, the output of step 1 at stage k - 1. So T iterations of the
// stages of an interior range [a, b) need only the stages [a - T, b + T) at the start: a window
// loaded once into shared memory, iterated T times there, and written back on its interior.
// The stages of the halo go wrong one per iteration from each open end of the window (the first
// stage lacks xbar from its left neighbour, the last one the iterates of its right neighbour;
// at the horizon's ends the window is closed and nothing goes wrong), so after T iterations
// exactly [a, b) is right. Stage data and iterates cross HBM once per T iterations instead of
// once per iteration, at the price of recomputing the halos.
//
// The stop test (Algorithm 1 step 5) needs c of every iteration over the whole instance, which a
// window does not see; c is summed over the interiors at the last iteration of each block of T,
// so an instance stops at the first multiple of T (or max_iters) where c <= eps. The accelerated
// iteration (steps 6-7) decides per iteration on c, so this schedule runs the plain one only.
// One CTA per window, a group of g lanes per stage (the resident kernel's per-stage code); the
// frame (items, grid barrier between blocks, compaction) is the lock-step one, with one frame
// iteration per block of T iterations.
#include <math.h>

#include "lockstep.cuh"
#include "products.cuh"

namespace pimpc {

namespace {

template <typename T>
using Args = ls::Args<T>;

constexpr int kTbThreads = 512;

struct TbPlan {
  int T;  // iterations per block
};

// Shared-memory regions (elements, 8-element aligned) of a window of L stages of one instance:
// stage blocks, two iterate buffers, xbar rows, du rows, the lane groups' scratch.
struct TbRegions {
  int offI, itb, offX, offD, offS, total;
};

__host__ __device__ inline int tb_group(int n) { return n <= 8 ? 8 : (n <= 16 ? 16 : 32); }

__host__ __device__ inline TbRegions tb_regions(int n, int W, int lti, int ts, int L) {
  const int nv = (n + 3) & ~3, n5p = ls::iter_stride_plain(n, ts);
  auto up = [](int v) { return (v + 7) / 8 * 8; };
  TbRegions R;
  R.offI = up((lti ? 2 : L) * W);
  R.itb = up(L * n5p);
  R.offX = R.offI + 2 * R.itb;
  R.offD = R.offX + up((L + 1) * nv);
  R.offS = R.offD + up(L * nv);
  R.total = R.offS + up((kTbThreads / tb_group(n)) * 4 * nv);
  return R;
}

// Steps 5 of Algorithm 1 for the plain iteration at the end of a block: the instance's last item
// adds up c and stops the instance on c <= eps, a non-finite c, or max_iters. Called by one thread.
template <typename T>
__device__ inline void finish_block(const Args<T> &a, int j, int blk, int iters, double part) {
  atomicAdd(&a.cacc[j], part);
  __threadfence();
  const int done = atomicAdd(&a.ndone[j], 1);
  if (done != a.nitems_inst[j] - 1) return;
  __threadfence();
  const double s = __longlong_as_double((long long)atomicExch((unsigned long long *)&a.cacc[j], 0ull));
  a.ndone[j] = 0;
  const double c = a.rho * s;
  InstState &st = a.st[j];
  st.iters = iters;
  st.c = c;
  int stop = 0;
  if (!isfinite(c)) {
    st.status = kNonFinite; stop = 1;
  } else if (c <= a.eps) {
    st.status = kConverged; stop = 1;
  } else if (iters >= a.max_iters) {
    st.status = kMaxIter; stop = 1;
  }
  a.coef[j] = 0.0;
  a.cprev[j] = c;
  if (stop) {
    a.stop[j] = 1;
    a.base[j] = (a.base[j] + blk + 1) % 3;  // the buffer holding the final iterate
    atomicSub(&a.ctl->active, 1);
    atomicExch(&a.ctl->stopped, 1);
  }
}

template <typename T>
__global__ void __launch_bounds__(kTbThreads) tb_kernel(Args<T> a, TbPlan pl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sRed[kTbThreads / 32];
  __shared__ int sItem, sOk;
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;
  const int lti = a.L.lti;
  const int nblk_total = (a.max_iters + pl.T - 1) / pl.T;

  int cl = 0;
  for (int blk = 0; blk < nblk_total; ++blk) {
    const int Tb = min(pl.T, a.max_iters - blk * pl.T);
    const int nact = *(volatile int *)&ctl->nlist[cl];
    for (;;) {
      if (tid == 0) sItem = atomicAdd(&ctl->queue[blk & 1], 1);
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
      const int g = tb_group(n), ngrp = nthreads / g, grp = tid / g, l = tid - grp * g;
      const int ncl = (g == 32 && n > 32) ? 2 : 1;
      const int nv = (n + 3) & ~3;
      const int n5p = ls::iter_stride_plain(n, (int)sizeof(T));
      const int W = a.L.W[j];
      const int ldg = odd_ld(n);
      const int oE = nx * ldg, oH = oE + nx, oM = oH + wrapped_size(n);
      const int lo = max(ka - Tb, 0), hi = min(kb + Tb, N), L = hi - lo;
      const unsigned gmask = g == 32 ? 0xffffffffu : (((1u << g) - 1u) << ((tid & 31) & ~(g - 1)));
      const TbRegions R = tb_regions(n, W, lti, (int)sizeof(T), L);
      T *B = sm;
      T *I[2] = {sm + R.offI, sm + R.offI + R.itb};
      T *X = sm + R.offX;  // row q: xbar_{lo + q}
      T *D = sm + R.offD;  // row q: du_{lo + q}
      T *scr = sm + R.offS + grp * 4 * nv;
      T *sW = scr, *sY = scr + nv, *sH = scr + 2 * nv, *sDU = scr + 3 * nv;
      const T rho = (T)a.rho;
      const T *qd = a.qd + a.L.off_n[j];
      const T *ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
      const int refstride = a.ref_per_stage ? n : 0;
      const T *lo_b = a.lo + a.L.off_n[j], *hi_b = a.hi + a.L.off_n[j];
      const int bse = a.base[j];
      const int64_t ib = a.L.Ni[j];
      const T *Ic = a.it[(bse + blk) % 3] + ib;
      T *In = a.it[(bse + blk + 1) % 3] + ib;

      // ---- the window: stage blocks, iterates, xbar_lo (exact only at the horizon's start) ----
      {
        const T *gblk = a.blk + a.L.blk[j];
        const int nbw = lti ? 2 * W : L * W;
        const int64_t from = lti ? 0 : (int64_t)lo * W;
        for (int e = tid; e < nbw; e += nthreads) B[e] = gblk[from + e];
        for (int e = tid; e < L * n5p; e += nthreads) I[0][e] = Ic[(int64_t)lo * n5p + e];
        for (int c = tid; c < nv; c += nthreads)
          X[c] = (lo == 0 && c < n) ? a.xb0[a.L.off_n[j] + c] : (T)0;
      }
      __syncthreads();
      int cur = 0;
      T cacc = (T)0;
      for (int t = 0; t < Tb; ++t) {
        const T *Ic_s = I[cur];
        T *In_s = I[cur ^ 1];
        // ---- phase 1: step 1 on every stage of the window ----
        for (int kb0 = lo; kb0 < hi; kb0 += ngrp) {
          const int k = kb0 + grp;
          const bool active = k < hi;
          const int kl = k - lo;
          const bool next_local = kl + 1 < L;  // the next stage is in the window
          const T *Gk = lti ? B : B + (int64_t)kl * W;
          const T *Gk1 = lti ? B : B + (int64_t)(next_local ? kl + 1 : kl) * W;
          const T *Hk = lti ? (B + ((k < N - 1) ? 0 : W)) : Gk;
          const T *hc = Ic_s + kl * n5p;
          const T *nc = hc + n5p;
          const bool with_y = k + 1 < N && next_local;  // else y = 0 (exact only when k = N - 1)
          T zh[2], thh[2];
          if (active) {
            for (int qq = 0; qq < ncl; ++qq) {
              const int c = l + 32 * qq;
              if (c < n) {
                zh[qq] = hc[c];
                thh[qq] = hc[2 * n + c];
                sW[c] = hc[n + c] - hc[3 * n + c];
                sY[c] = with_y ? nc[c] - nc[n + c] + nc[4 * n + c] - (c < nx ? Gk1[oE + c] : (T)0)
                               : (T)0;
              }
            }
          }
          __syncwarp(gmask);
          if (active && l < nu) sH[l] = sW[nx + l] + dot_col(Gk + nx + l, ldg, sW, nx);
          __syncwarp(gmask);
          if (active && l < nu) {
            const T du = sym_wrapped(Gk + oM, sH, nu, l);
            sDU[l] = du;
            D[kl * nv + l] = du;
          }
          __syncwarp(gmask);
          if (active) {
            for (int qq = 0; qq < ncl; ++qq) {
              const int c = l + 32 * qq;
              if (c < n) {
                T acc = (T)0;
                if (with_y) {
                  acc = dot_col(Gk1 + c, ldg, sY, nx);
                  if (c >= nx) acc += sY[c];
                }
                const T rf = ref ? ref[(int64_t)k * refstride + c] : (T)0;
                sH[c] = qd[c] * rf + rho * (zh[qq] - thh[qq] + acc);
              }
            }
          }
          __syncwarp(gmask);
          if (active)
            for (int qq = 0; qq < ncl; ++qq) {
              const int c = l + 32 * qq;
              if (c < n) X[(kl + 1) * nv + c] = sym_wrapped(Hk + oH, sH, n, c);
            }
          __syncwarp(gmask);
        }
        __syncthreads();
        // ---- phase 2: steps 2-4 on every stage of the window (c on the interior, last iteration) ----
        const bool lastit = t == Tb - 1;
        for (int kb0 = lo; kb0 < hi; kb0 += ngrp) {
          const int k = kb0 + grp;
          if (k >= hi) continue;
          const int kl = k - lo;
          const bool inner = lastit && k >= ka && k < kb;
          const T *Gk = lti ? B : B + (int64_t)kl * W;
          const T *hc = Ic_s + kl * n5p;
          const T *xk = X + kl * nv, *xk1 = X + (kl + 1) * nv, *du = D + kl * nv;
          T *o = In_s + kl * n5p;
          for (int qq = 0; qq < ncl; ++qq) {
            const int c = l + 32 * qq;
            if (c >= n) continue;
            const T zh = hc[c], vh = hc[n + c], thh = hc[2 * n + c], beh = hc[3 * n + c];
            const T lah = hc[4 * n + c];
            T ax, bd, ee;
            if (c < nx) {
              const T *row = Gk + c * ldg;
              ax = dot_col(row, 1, xk, n);
              bd = dot_col(row + nx, 1, du, nu);
              ee = Gk[oE + c];
            } else {
              ax = xk[c]; bd = du[c - nx]; ee = (T)0;
            }
            const T xn = xk1[c];
            const T gam = bd + beh - ax - ee + lah;
            const T w = ((T)2 * (xn + thh + ax + ee - lah) + gam) / (T)3;
            const T z = w < lo_b[c] ? lo_b[c] : (w > hi_b[c] ? hi_b[c] : w);
            const T v = (T)0.5 * (z + gam);
            const T th = thh + xn - z;
            const T be = beh + bd - v;
            const T la = lah + z - ax - v - ee;
            if (inner) {
              const T d1 = th - thh, d2 = be - beh, d3 = la - lah, d4 = z - zh, d5 = v - vh;
              const T d6 = d4 - d5;
              cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
            }
            o[c] = z; o[n + c] = v; o[2 * n + c] = th; o[3 * n + c] = be; o[4 * n + c] = la;
          }
        }
        __syncthreads();
        cur ^= 1;
      }
      // ---- the interior back to HBM ----
      {
        const int off = (ka - lo) * n5p, cnt = (kb - ka) * n5p;
        for (int e = tid; e < cnt; e += nthreads) In[(int64_t)ka * n5p + e] = I[cur][off + e];
      }
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if ((tid & 31) == 0) sRed[tid >> 5] = (double)cacc;
      __syncthreads();
      if (tid == 0) {
        double part = 0.0;
        for (int w = 0; w < (nthreads >> 5); ++w) part += sRed[w];
        __threadfence();  // the interior's iterates before the instance's completion count
        finish_block(a, j, blk, blk * pl.T + Tb, part);
      }
      __syncthreads();
    }
    if (blockIdx.x == 0 && tid == 0) ctl->queue[(blk + 1) & 1] = 0;
    if (!ls::grid_sync(ctl, nblocks, &sOk)) break;
    if (*(volatile int *)&ctl->active <= 0) break;
    if (!ls::compact(a, cl, nact, &sOk, reinterpret_cast<int *>(sRed))) break;
  }
}

}  // namespace

int tb_threads() { return kTbThreads; }

// Shared-memory words of a window of S stages (one instance).
int64_t tb_window_words(int nx, int nu, int W, int lti, int precision, int S) {
  return tb_regions(nx + nu, W, lti, precision == 0 ? 4 : 8, S).total;
}

size_t tb_static_smem(int precision) {
  cudaFuncAttributes fa{};
  const cudaError_t rc = precision == 0 ? cudaFuncGetAttributes(&fa, tb_kernel<float>)
                                        : cudaFuncGetAttributes(&fa, tb_kernel<double>);
  return rc == cudaSuccess ? fa.sharedSizeBytes : 1024;
}

cudaError_t tb_configure(int precision, size_t smem, int *blocks_per_sm) {
  cudaError_t rc;
  if (precision == 0) {
    rc = cudaFuncSetAttribute(tb_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tb_kernel<float>, kTbThreads, smem);
  }
  rc = cudaFuncSetAttribute(tb_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (rc != cudaSuccess) return rc;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tb_kernel<double>, kTbThreads, smem);
}

cudaError_t launch_tb(const AdmmLaunch &s, int precision, int T, size_t smem, cudaStream_t stream) {
  TbPlan pl;
  pl.T = T;
  if (precision == 0) {
    ls::Args<float> a = ls::make_args<float>(s);
    void *params[] = {&a, &pl};
    return ls::launch_sequence<float>(s, a, (const void *)tb_kernel<float>, params, smem, stream);
  }
  ls::Args<double> a = ls::make_args<double>(s);
  void *params[] = {&a, &pl};
  return ls::launch_sequence<double>(s, a, (const void *)tb_kernel<double>, params, smem, stream);
}

}  // namespace pimpc

// admm_res.cu -- Algorithm 1 with every instance resident on chip: one CTA, or a thread-block
// cluster of C CTAs, per instance (schedule family 3).
//
// The lock-step kernels stream the stage data from HBM every iteration and separate iterations
// by a grid-wide barrier (global atomics); for a single instance or a small batch that barrier,
// not the arithmetic, sets the time per iteration. Here instance j is solved by cluster j alone:
// CTA r of the cluster holds stages [r N / C, (r + 1) N / C) -- their stage blocks (plus the
// block of the next stage, whose G and e its last stage reads), three rotating iterate buffers,
// the xbar rows and du of its slice -- in shared memory for the whole solve, loaded once.
// Per iteration (the phases of the lane-group kernel, a group of g lanes per stage):
//   phase 1: du_k and xbar_{k+1} = H_k h_k for the slice; the hats of the first stage of the next
//            slice are read from the neighbouring CTA's shared memory (distributed shared memory);
//   cluster barrier; xbar of the slice's first stage is copied from the previous CTA;
//   phase 2: the (v, z) update, the duals and the CTA's share of c;
//   cluster barrier; every CTA adds the C shares in rank order and applies steps 5-7 itself
//   (identical inputs and order, hence identical decisions: every CTA of the cluster runs the
//   same number of iterations, so the hardware cluster barriers always complete).
// The final iterate is written back to the solver's iterate buffer; nothing crosses a cluster.
#include <cooperative_groups.h>
#include <math.h>

#include "lockstep.cuh"
#include "products.cuh"

namespace cg = cooperative_groups;

namespace pimpc {

namespace {

template <typename T>
using Args = ls::Args<T>;

// Shared-memory regions of one CTA (elements of T, 16-byte aligned offsets).
struct ResPlan {
  int C;          // CTAs per instance (cluster size)
  int offI, itb;  // iterate buffers: 3 of itb elements
  int offX, offD, offS;
};

__host__ __device__ inline int res_group(int n) { return n <= 8 ? 8 : (n <= 16 ? 16 : 32); }
__host__ __device__ inline int res_stride(int n, int tsize) {
  const int q = 16 / tsize;
  return (5 * n + q - 1) / q * q;
}

// kMinCtas: the CTAs of 256 threads per SM that the registers are capped for (0: no cap beyond
// the block size, the default). A batch of many small instances (more CTAs than the SMs hold at
// once) runs the variant capped for 4 in FP32 (64 registers, no spills): fewer waves. A cluster
// that spans one instance keeps the default, whose larger register budget shortens each
// iteration's critical path.
template <typename T, int kMinCtas>
__global__ void __launch_bounds__(256, kMinCtas) resident_kernel(Args<T> a, ResPlan pl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double sPart;
  __shared__ double sRed[8];
  __shared__ int sStop;
  __shared__ double sCoef;
  T *sm = reinterpret_cast<T *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int C = pl.C;
  const int r = (int)cl.block_rank();
  const int j = blockIdx.x / C;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
  const int g = res_group(n), ngrp = nthreads / g, grp = tid / g, l = tid - grp * g;
  const int ncl = (g == 32 && n > 32) ? 2 : 1;
  const int nv = (n + 3) & ~3;
  const int n5p = res_stride(n, (int)sizeof(T));
  const int W = a.L.W[j];
  const int ldg = odd_ld(n);
  const int oE = nx * ldg, oH = oE + nx, oM = oH + wrapped_size(n);
  const int lti = a.L.lti;
  const int k0 = (int)((int64_t)r * N / C), k1 = (int)((int64_t)(r + 1) * N / C), L = k1 - k0;
  const int Lprev = k0 - (int)((int64_t)(r - 1) * N / C);  // slice length of CTA r-1 (r > 0)
  const unsigned gmask = g == 32 ? 0xffffffffu : (((1u << g) - 1u) << ((tid & 31) & ~(g - 1)));
  T *B = sm;
  T *I[3] = {sm + pl.offI, sm + pl.offI + pl.itb, sm + pl.offI + 2 * pl.itb};
  T *X = sm + pl.offX;   // row q: xbar_{k0 + q}
  T *D = sm + pl.offD;   // row q: du_{k0 + q}
  T *scr = sm + pl.offS + grp * 4 * nv;
  T *sW = scr, *sY = scr + nv, *sH = scr + 2 * nv, *sDU = scr + 3 * nv;
  const T rho = (T)a.rho;
  const T *qd = a.qd + a.L.off_n[j];
  const T *ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
  const int refstride = a.ref_per_stage ? n : 0;
  const T *lo = a.lo + a.L.off_n[j], *hi = a.hi + a.L.off_n[j];

  // ---- load the slice (once) ----
  {
    const T *gblk = a.blk + a.L.blk[j];
    const int nblk = lti ? 2 : (k1 < N ? L + 1 : L);  // plus the next stage's block
    const int64_t from = lti ? 0 : (int64_t)k0 * W;
    for (int e = tid; e < nblk * W; e += nthreads) B[e] = gblk[from + e];
    const T *git = a.it[a.base[j]] + a.L.Ni[j] + (int64_t)k0 * n5p;
    for (int e = tid; e < L * n5p; e += nthreads) I[0][e] = git[e];
    if (r == 0)
      for (int c = tid; c < n; c += nthreads) X[c] = a.xb0[a.L.off_n[j] + c];
  }
  double cprev = 1.0, coef = 0.0;
  int streak = 0;  // consecutive momentum steps since the last restart
  int momentum = 0, status = kMaxIter, iters = 0;
  double cval = 0.0;
  double cbest = INFINITY;  // stall test: best c so far, the iteration that set it, and the
  int itbest = 0, itfirst = -1;  // first iteration with c <= stall_below
  int cur = 0, prv = 2, nw = 1;
  cl.sync();

  for (int it = 0; it < a.max_iters; ++it) {
    const T f = (T)coef;
    const bool use_prev = coef != 0.0;
    const T *Ic = I[cur], *Ip = I[prv];
    const T *Rc = nullptr, *Rp = nullptr;  // the next CTA's current and previous iterates
    if (r + 1 < C) {
      Rc = cl.map_shared_rank(I[cur], r + 1);
      Rp = cl.map_shared_rank(I[prv], r + 1);
    }
    // ---- phase 1: step 1 ----
    for (int kb = k0; kb < k1; kb += ngrp) {
      const int k = kb + grp;
      const bool active = k < k1;
      const int kl = k - k0;
      const T *Gk = lti ? B : B + (int64_t)kl * W;
      const T *Gk1 = lti ? B : B + (int64_t)(kl + 1) * W;
      const T *Hk = lti ? (B + ((k < N - 1) ? 0 : W)) : Gk;
      const T *hc = Ic + kl * n5p, *hp = Ip + kl * n5p;
      T zh[2], thh[2];
      if (active) {
        const bool next_local = kl + 1 < L;
        const T *nc = next_local ? hc + n5p : Rc, *np = next_local ? hp + n5p : Rp;
        for (int qq = 0; qq < ncl; ++qq) {
          const int c = l + 32 * qq;
          if (c < n) {
            T cz = hc[c], cv = hc[n + c], ct = hc[2 * n + c], cb = hc[3 * n + c];
            if (use_prev) {
              cz += f * (cz - hp[c]);
              cv += f * (cv - hp[n + c]);
              ct += f * (ct - hp[2 * n + c]);
              cb += f * (cb - hp[3 * n + c]);
            }
            zh[qq] = cz;
            thh[qq] = ct;
            sW[c] = cv - cb;
            T y = (T)0;
            if (k + 1 < N) {
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
      __syncwarp(gmask);
      if (active && l < nu) sH[l] = sW[nx + l] + dot_col(Gk + nx + l, ldg, sW, nx);  // B_k^T w_x + w_u
      __syncwarp(gmask);
      if (active && l < nu) {
        const T du = sym_wrapped(Gk + oM, sH, nu, l);  // du_k = M_k t
        sDU[l] = du;
        D[kl * nv + l] = du;
      }
      __syncwarp(gmask);
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
      __syncwarp(gmask);
      if (active)
        for (int qq = 0; qq < ncl; ++qq) {
          const int c = l + 32 * qq;
          if (c < n) X[(kl + 1) * nv + c] = sym_wrapped(Hk + oH, sH, n, c);  // xbar_{k+1} = H_k h_k
        }
      __syncwarp(gmask);
    }
    cl.sync();
    if (r > 0) {  // xbar_{k0}, computed by the previous CTA's last stage
      const T *px = cl.map_shared_rank(X, r - 1) + Lprev * nv;
      for (int c = tid; c < n; c += nthreads) X[c] = px[c];
    }
    __syncthreads();

    // ---- phase 2: steps 2-4 ----
    T cacc = (T)0;
    for (int kb = k0; kb < k1; kb += ngrp) {
      const int k = kb + grp;
      if (k >= k1) continue;
      const int kl = k - k0;
      const T *Gk = lti ? B : B + (int64_t)kl * W;
      const T *hc = Ic + kl * n5p, *hp = Ip + kl * n5p;
      const T *xk = X + kl * nv, *xk1 = X + (kl + 1) * nv, *du = D + kl * nv;
      T *o = I[nw] + kl * n5p;
      for (int qq = 0; qq < ncl; ++qq) {
        const int c = l + 32 * qq;
        if (c >= n) continue;
        T zh = hc[c], vh = hc[n + c], thh = hc[2 * n + c], beh = hc[3 * n + c], lah = hc[4 * n + c];
        if (use_prev) {
          zh += f * (zh - hp[c]);
          vh += f * (vh - hp[n + c]);
          thh += f * (thh - hp[2 * n + c]);
          beh += f * (beh - hp[3 * n + c]);
          lah += f * (lah - hp[4 * n + c]);
        }
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
        const T z = w < lo[c] ? lo[c] : (w > hi[c] ? hi[c] : w);
        const T v = (T)0.5 * (z + gam);
        const T th = thh + xn - z;
        const T be = beh + bd - v;
        const T la = lah + z - ax - v - ee;
        const T d1 = th - thh, d2 = be - beh, d3 = la - lah, d4 = z - zh, d5 = v - vh, d6 = d4 - d5;
        cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
        o[c] = z; o[n + c] = v; o[2 * n + c] = th; o[3 * n + c] = be; o[4 * n + c] = la;
      }
    }
    for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
    if ((tid & 31) == 0) sRed[tid >> 5] = (double)cacc;
    __syncthreads();
    if (tid == 0) {
      double part = 0.0;
      for (int w = 0; w < (nthreads >> 5); ++w) part += sRed[w];
      sPart = part;
    }
    cl.sync();

    // ---- steps 4-7, taken identically by every CTA of the cluster ----
    // Lane q of warp 0 reads the share of CTA q (one round of remote loads); the shares are
    // added by a fixed butterfly, so lane 0 holds the same sum in every CTA.
    if (tid < 32) {
      double s = tid < C ? *cl.map_shared_rank(&sPart, tid) : 0.0;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (tid == 0) sRed[0] = s;
    }
    __syncwarp();
    if (tid == 0) {
      const double s = sRed[0];
      const double c = a.rho * s;
      cval = c;
      iters = it + 1;
      int stop = 0;
      if (!isfinite(c)) {
        status = kNonFinite; stop = 1;
      } else if (c <= a.eps) {
        status = kConverged; stop = 1;
      } else if (a.stall_win > 0 && c <= a.stall_below && !(c < a.stall_fac * cbest) &&
                 (double)(it - itbest) >=
                     fmax((double)a.stall_win, a.stall_rel * (double)(itfirst < 0 ? it : itfirst))) {
        status = kStalled; stop = 1;
      } else if (it + 1 >= a.max_iters) {
        status = kMaxIter; stop = 1;
      } else {
        int take = 0;
        if (a.accel) {
          if (a.mask && it < a.mask_len) take = a.mask[(int64_t)j * a.mask_len + it] != 0;
          else take = c <= a.eta * cprev;
        }
        if (take) {  // (alpha_m - 1) / alpha_{m+1}, alpha_0 = 1, from the precomputed table
          coef = a.coef_tab[streak];
          if (streak > 0) momentum += 1;
          ++streak;
        } else {
          streak = 0;
          coef = 0.0;
        }
        cprev = c;
      }
      if (c <= a.stall_below) {
        if (itfirst < 0) itfirst = it;
        if (c < a.stall_fac * cbest) {
          cbest = c;
          itbest = it;
        }
      }
      sStop = stop;
      sCoef = coef;
    }
    __syncthreads();
    coef = sCoef;
    const int t3 = prv;
    prv = cur;
    cur = nw;
    nw = t3;
    if (sStop) break;
  }
  // Final iterate -> the solver's iterate buffer (the one the starting iterate came from).
  {
    T *git = a.it[a.base[j]] + a.L.Ni[j] + (int64_t)k0 * n5p;
    for (int e = tid; e < L * n5p; e += nthreads) git[e] = I[cur][e];
  }
  if (r == 0 && tid == 0) {
    InstState s;
    s.iters = iters;
    s.status = status;
    s.momentum = momentum;
    s.pad = 0;
    s.c = cval;
    a.st[j] = s;
    a.stop[j] = 1;
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename T>
cudaError_t launch_t(const AdmmLaunch &s, const ResPlan &pl, size_t smem, cudaStream_t stream) {
  Args<T> a = ls::make_args<T>(s);
  cudaError_t rc = cudaMemcpyAsync(s.old_base, s.base, sizeof(int) * s.L.batch,
                                   cudaMemcpyDeviceToDevice, stream);
  if (rc != cudaSuccess) return rc;
  const int n_init = s.L.batch > s.nitems ? s.L.batch : s.nitems;
  ls::solve_init_kernel<T><<<(n_init + 255) / 256, 256, 0, stream>>>(a, s.warm);
  if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
  if (s.warm != 1) {
    ls::prepare_kernel<T><<<dim3(8, s.L.batch), 256, 0, stream>>>(a, s.warm, s.old_base);
    if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
  }
  if (s.max_iters > 0) {
    const void *kernel = (const void *)resident_kernel<T, 0>;
    if constexpr (sizeof(T) == 4) {
      int dev = 0, nsm = 0;
      if ((rc = cudaGetDevice(&dev)) != cudaSuccess) return rc;
      if ((rc = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return rc;
      if ((int64_t)s.L.batch * pl.C > 2 * (int64_t)nsm) kernel = (const void *)resident_kernel<T, 4>;
    }
    rc = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    if (pl.C > 8) {
      rc = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (rc != cudaSuccess) return rc;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s.L.batch * pl.C);
    cfg.blockDim = dim3(s.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pl.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ResPlan plc = pl;
    void *params[] = {&a, &plc};
    rc = cudaLaunchKernelExC(&cfg, kernel, params);
    if (rc != cudaSuccess) return rc;
  }
  ls::output_kernel<T><<<dim3(4, s.L.batch), 256, 0, stream>>>(a, s.u_out, s.x_out);
  return cudaGetLastError();
}

// tab[m] = (alpha_m - 1) / alpha_{m+1} with alpha_0 = 1, alpha_{m+1} = (1 + sqrt(1 + 4 alpha_m^2))
// / 2: the momentum factor of Algorithm 1 step 6 after m consecutive momentum steps.
__global__ void coef_table_kernel(double *tab, int len) {
  double al = 1.0;
  for (int m = 0; m < len; ++m) {
    const double an = 0.5 + 0.5 * sqrt(1.0 + 4.0 * al * al);
    tab[m] = (al - 1.0) / an;
    al = an;
  }
}

}  // namespace

cudaError_t launch_coef_table(double *tab, int len, cudaStream_t stream) {
  coef_table_kernel<<<1, 1, 0, stream>>>(tab, len);
  return cudaGetLastError();
}

int res_threads(int precision) { return precision == 0 ? 256 : 128; }

// Plans the shared memory of one CTA for a cluster of C CTAs per instance; returns the bytes
// needed (0 if some instance has fewer than C stages).
size_t res_plan(int batch, const int *nx, const int *nu, const int *N, const int *W, int lti,
                int precision, int threads, int C, int *plan) {
  const int ts = precision == 0 ? 4 : 8;
  int64_t blk = 0, itb = 0, xw = 0, dw = 0, sw = 0;
  for (int j = 0; j < batch; ++j) {
    if (N[j] < C) return 0;
    const int n = nx[j] + nu[j];
    const int L = (N[j] + C - 1) / C;
    const int nv = (n + 3) & ~3;
    const int n5p = res_stride(n, ts);
    blk = std::max<int64_t>(blk, (int64_t)(lti ? 2 : L + 1) * W[j]);
    itb = std::max<int64_t>(itb, (int64_t)L * n5p);
    xw = std::max<int64_t>(xw, (int64_t)(L + 1) * nv);
    dw = std::max<int64_t>(dw, (int64_t)L * nv);
    sw = std::max<int64_t>(sw, (int64_t)(threads / res_group(n)) * 4 * nv);
  }
  auto up = [](int64_t v) { return (v + 7) / 8 * 8; };
  const int64_t offI = up(blk), offX = offI + 3 * up(itb), offD = offX + up(xw), offS = offD + up(dw);
  const int64_t total = offS + up(sw);
  plan[0] = C;
  plan[1] = (int)offI;
  plan[2] = (int)up(itb);
  plan[3] = (int)offX;
  plan[4] = (int)offD;
  plan[5] = (int)offS;
  return (size_t)total * ts;
}

cudaError_t launch_resident(const AdmmLaunch &s, int precision, const int *plan, size_t smem,
                            cudaStream_t stream) {
  ResPlan pl;
  pl.C = plan[0];
  pl.offI = plan[1];
  pl.itb = plan[2];
  pl.offX = plan[3];
  pl.offD = plan[4];
  pl.offS = plan[5];
  return precision == 0 ? launch_t<float>(s, pl, smem, stream) : launch_t<double>(s, pl, smem, stream);
}

}  // namespace pimpc

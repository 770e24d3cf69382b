// admm_gemm.cu -- Algorithm 1 for stage-invariant instances as dense contractions (schedule
// family 4).
//
// When A, B, e (and so G, M and, except for the last stage, H) are the same at every stage, the
// per-stage products of a block of consecutive stages share their matrix: with the stages as
// columns they are matrix-matrix products with K, M <= 64 and one column per stage,
//   T  = B^T W_x + W_u          W   = Vhat - Betahat             (nu x nx) (nx x L)
//   DU = M T                                                     (nu x nu) (nu x L)
//   Hh = qbar ref + rho (Zhat - Thetahat + G^T Y_x + [0; Y_u])   (n x nx)  (nx x (L+1))
//   Xb = H Hh  (xbar_{k+1} of every column; the last stage uses H_{N-1})  (n x n) (n x (L+1))
//   AX = G Xb(shifted by one column),  BD = B DU                  (nx x n)  (n x L)
// followed by the elementwise steps 2-3 and the share of c. Each product runs as a
// register-tiled contraction on the CUDA cores in FP32 (or FP64): every thread accumulates a
// 4 x 4 tile of outputs over K, sixteen multiply-adds per eight operand loads. (The tensor
// cores' TF32/BF16 inputs would not keep the iterations at FP32 accuracy; FP64 tensor rates are
// low on this part.)
//
// Work items are runs of consecutive stage blocks (LB stages each) of one instance, in the
// lock-step frame of lockstep.cuh (grid barrier between iterations, steps 5-7 in the pass over
// the instances after it). A block reads the hats of one stage more on each side
// (the xbar of its first stage is recomputed from stage a-1, the y of its last stage needs stage
// b), so items of one iteration are independent. The instance's matrices are expanded from the
// stage block into shared memory once per item (from L2: they are shared by all items of the
// instance); one CTA of 512 threads per SM leaves room for blocks of about 90 stages at n = 64.
#include <math.h>

#include "lockstep.cuh"

namespace pimpc {

namespace {

template <typename T>
using Args = ls::Args<T>;

constexpr int kGemmThreads = 512;

struct GemmPlan {
  int LB;          // stages per block (an item holds one or more consecutive blocks)
  int LP;          // columns of a work matrix (LB + 2)
  int nP, nxP, nuP;  // padded row lengths of the matrices (maxima over the batch)
  // shared-memory offsets (elements of T)
  int oG, oGT, oH, oM, oB, oE, oHAT, oX1, oX2, oT, oDU, total;
};

template <typename T>
__device__ __forceinline__ T wrapped_at(const T *Wp, int m, int r, int c) {
  int d = c - r;
  if (d < 0) d += m;
  return (2 * d <= m) ? Wp[d * m + r] : Wp[(m - d) * m + c];
}

// out(m, col, acc) for m < M and col < NC with acc = sum_{k < K} AT[k lda + m] B[k ldb + col]:
// thread t owns rows tm, tm + SM, tm + 2 SM, tm + 3 SM and columns tn, tn + SN, ... (SM, SN =
// ceil(M / 4), ceil(NC / 4)), so consecutive threads read consecutive words of AT.
template <typename T, typename F>
__device__ __forceinline__ void gemm_tiles(const T *AT, int lda, const T *B, int ldb, int M, int K,
                                           int NC, F out) {
  const int SM = (M + 3) >> 2, SN = (NC + 3) >> 2;
  for (int t = threadIdx.x; t < SM * SN; t += blockDim.x) {
    const int tm = t % SM, tn = t / SM;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] = (T)0;
    bool mv[4], cv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      mv[i] = tm + i * SM < M;
      cv[i] = tn + i * SN < NC;
    }
    for (int k = 0; k < K; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = mv[i] ? AT[k * lda + tm + i * SM] : (T)0;
        bv[i] = cv[i] ? B[k * ldb + tn + i * SN] : (T)0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] += av[i] * bv[q];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (mv[i] && cv[q]) out(tm + i * SM, tn + q * SN, acc[i][q]);
  }
}

// Two contractions into the same outputs: acc1 over (AT1, B1, K1) and acc2 over (AT2, B2, K2).
template <typename T, typename F>
__device__ __forceinline__ void gemm_tiles2(const T *AT1, int lda1, const T *B1, int ldb1, int K1,
                                            const T *AT2, int lda2, const T *B2, int ldb2, int K2,
                                            int M, int NC, F out) {
  const int SM = (M + 3) >> 2, SN = (NC + 3) >> 2;
  for (int t = threadIdx.x; t < SM * SN; t += blockDim.x) {
    const int tm = t % SM, tn = t / SM;
    T a1[4][4], a2[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) a1[i][q] = a2[i][q] = (T)0;
    bool mv[4], cv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      mv[i] = tm + i * SM < M;
      cv[i] = tn + i * SN < NC;
    }
    for (int k = 0; k < K1; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = mv[i] ? AT1[k * lda1 + tm + i * SM] : (T)0;
        bv[i] = cv[i] ? B1[k * ldb1 + tn + i * SN] : (T)0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) a1[i][q] += av[i] * bv[q];
    }
    for (int k = 0; k < K2; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = mv[i] ? AT2[k * lda2 + tm + i * SM] : (T)0;
        bv[i] = cv[i] ? B2[k * ldb2 + tn + i * SN] : (T)0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) a2[i][q] += av[i] * bv[q];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (mv[i] && cv[q]) out(tm + i * SM, tn + q * SN, a1[i][q], a2[i][q]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(Args<T> a, GemmPlan pl) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int sItem, sOk;
  __shared__ double sRed[kGemmThreads / 32];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;
  T *Gs = sm + pl.oG, *GT = sm + pl.oGT, *Hs = sm + pl.oH, *Ms = sm + pl.oM, *Bs = sm + pl.oB;
  T *Es = sm + pl.oE, *HAT = sm + pl.oHAT, *X1 = sm + pl.oX1, *X2 = sm + pl.oX2;
  T *Ts = sm + pl.oT, *DU = sm + pl.oDU;
  const int LP = pl.LP, nP = pl.nP, nxP = pl.nxP, nuP = pl.nuP;

  int cl = 0;
  for (int it = 0; it < a.max_iters; ++it) {
    const int nact = *(volatile int *)&ctl->nlist[cl];
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
      const int ia = a.item_a[item], ib_end = a.item_b[item];
      const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
      const int W = a.L.W[j];
      const int ldg = odd_ld(n);
      const int oE = nx * ldg, oH = oE + nx, oM = oH + wrapped_size(n);
      const int n5p = ls::iter_stride_plain(n, (int)sizeof(T));
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
      T cacc = (T)0;

      // ---- the instance's matrices (once per item) ----
      for (int e = tid; e < nx * n; e += nthreads) {
        const int r = e / n, c = e - r * n;
        const T gv = blk[r * ldg + c];
        Gs[r * nP + c] = gv;
        GT[c * nxP + r] = gv;
        if (c >= nx) Bs[r * nuP + (c - nx)] = gv;
      }
      for (int e = tid; e < nx; e += nthreads) Es[e] = blk[oE + e];
      for (int e = tid; e < n * n; e += nthreads) {
        const int r = e / n, c = e - r * n;
        Hs[r * nP + c] = wrapped_at(blk + oH, n, r, c);
      }
      for (int e = tid; e < nu * nu; e += nthreads) {
        const int r = e / nu, c = e - r * nu;
        Ms[r * nuP + c] = wrapped_at(blk + oM, nu, r, c);
      }
      // ---- blocks of LB stages [ka, kb) of the item, one after the other ----
      for (int ka = ia; ka < ib_end; ka += pl.LB) {
      const int kb = min(ib_end, ka + pl.LB), L = kb - ka;
      const int NC = L + 2;  // columns: stages ka-1 .. kb
      __syncthreads();       // the previous block's readers are done with the work matrices
      for (int e = tid; e < 5 * n * NC; e += nthreads) {
        const int col = e / (5 * n), bc = e - col * 5 * n;
        const int s = ka - 1 + col;
        T v = (T)0;
        if (s >= 0 && s < N) {
          v = Ic[(int64_t)s * n5p + bc];
          if (use_prev) v += f * (v - Ip[(int64_t)s * n5p + bc]);
        }
        const int b = bc / n, c = bc - b * n;
        HAT[(b * nP + c) * LP + col] = v;
      }
      __syncthreads();
      auto hat = [&](int b, int c, int col) -> T { return HAT[(b * nP + c) * LP + col]; };

      // ---- step 1: W = Vhat - Betahat (own columns 1..L), T = B^T W_x + W_u, DU = M T ----
      for (int e = tid; e < n * L; e += nthreads) {
        const int c = e / L, col = 1 + e - (e / L) * L;
        X1[c * LP + col] = hat(1, c, col) - hat(3, c, col);
      }
      __syncthreads();
      gemm_tiles(Bs, nuP, X1 + 1, LP, nu, nx, L, [&](int qq, int cc, T acc) {
        Ts[qq * LP + 1 + cc] = acc + X1[(nx + qq) * LP + 1 + cc];
      });
      __syncthreads();
      gemm_tiles(Ms, nuP, Ts + 1, LP, nu, nu, L, [&](int qq, int cc, T acc) {
        DU[qq * LP + 1 + cc] = acc;
      });
      // Y_k = Zhat_{k+1} - Vhat_{k+1} - ebar + Lambdahat_{k+1}, columns 0..L (stages ka-1..kb-1)
      for (int e = tid; e < n * (L + 1); e += nthreads) {
        const int c = e / (L + 1), col = e - c * (L + 1);
        const int s = ka - 1 + col;
        T y = (T)0;
        if (s + 1 < N)
          y = hat(0, c, col + 1) - hat(1, c, col + 1) + hat(4, c, col + 1) - (c < nx ? Es[c] : (T)0);
        X1[c * LP + col] = y;
      }
      __syncthreads();
      // Hh = qbar ref + rho (Zhat - Thetahat + G^T Y_x + [0; Y_u])
      gemm_tiles(Gs, nP, X1, LP, n, nx, L + 1, [&](int c, int col, T acc) {
        const int s = ka - 1 + col;
        if (c >= nx) acc += X1[c * LP + col];
        const T rf = ref ? ref[(int64_t)(s < 0 ? 0 : s) * refstride + c] : (T)0;
        X2[c * LP + col] = qd[c] * rf + rho * (hat(0, c, col) - hat(2, c, col) + acc);
      });
      __syncthreads();
      // Xb = H Hh (xbar_{k+1} of stage ka-1+col); column 0 of the first item is xbar_0
      gemm_tiles(Hs, nP, X2, LP, n, n, L + 1, [&](int c, int col, T acc) {
        X1[c * LP + col] = acc;
      });
      __syncthreads();
      if (ka == 0)
        for (int c = tid; c < n; c += nthreads) X1[c * LP] = a.xb0[a.L.off_n[j] + c];
      if (kb == N) {  // the terminal stage: H_{N-1} (second block of the instance)
        const int col = L;
        for (int c = tid; c < n; c += nthreads) {
          T s = (T)0;
          for (int kk = 0; kk < n; ++kk) s += wrapped_at(blk + W + oH, n, c, kk) * X2[kk * LP + col];
          X1[c * LP + col] = s;
        }
      }
      __syncthreads();

      // ---- steps 2-4 for stages ka..kb-1 (own columns 1..L) ----
      auto update = [&](int r, int col, T ax, T bd) {
        const int s = ka - 1 + col;
        const T ee = r < nx ? Es[r] : (T)0;
        const T zh = hat(0, r, col), vh = hat(1, r, col), thh = hat(2, r, col);
        const T beh = hat(3, r, col), lah = hat(4, r, col);
        const T xn = X1[r * LP + col];
        const T gam = bd + beh - ax - ee + lah;
        const T w = ((T)2 * (xn + thh + ax + ee - lah) + gam) / (T)3;
        const T z = w < lo[r] ? lo[r] : (w > hi[r] ? hi[r] : w);
        const T v = (T)0.5 * (z + gam);
        const T th = thh + xn - z;
        const T be = beh + bd - v;
        const T la = lah + z - ax - v - ee;
        const T d1 = th - thh, d2 = be - beh, d3 = la - lah, d4 = z - zh, d5 = v - vh, d6 = d4 - d5;
        cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
        T *o = In + (int64_t)s * n5p;
        o[r] = z; o[n + r] = v; o[2 * n + r] = th; o[3 * n + r] = be; o[4 * n + r] = la;
      };
      // x-part: AX = G xbar_k (column col-1), BD = B du_k
      gemm_tiles2(GT, nxP, X1, LP, n, GT + nx * nxP, nxP, DU + 1, LP, nu, nx, L,
                  [&](int r, int cc, T ax, T bd) { update(r, cc + 1, ax, bd); });
      // u-part: ax = xbar_k,u, bd = du_k
      for (int e = tid; e < nu * L; e += nthreads) {
        const int q2 = e / L, cc = e - q2 * L;
        update(nx + q2, cc + 1, X1[(nx + q2) * LP + cc], DU[q2 * LP + cc + 1]);
      }
      }  // blocks of the item
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if ((tid & 31) == 0) sRed[tid >> 5] = (double)cacc;
      __syncthreads();
      if (tid == 0) {
        double part = 0.0;
        for (int w2 = 0; w2 < (nthreads >> 5); ++w2) part += sRed[w2];
        a.cpart[item] = part;  // steps 5-7 run in the pass after the barrier
      }
    }
    if (blockIdx.x == 0 && tid == 0) ctl->queue[(it + 1) & 1] = 0;
    if (!ls::grid_sync(ctl, nblocks, &sOk)) break;
    if (!ls::finish_pass(a, it, cl, nblocks, &sOk)) break;
    if (*(volatile int *)&ctl->active <= 0) break;
    if (!ls::compact(a, cl, nact, &sOk, reinterpret_cast<int *>(sRed))) break;
  }
}

template <typename T>
cudaError_t launch_t(const AdmmLaunch &s, const GemmPlan &pl, cudaStream_t stream) {
  Args<T> a = ls::make_args<T>(s);
  GemmPlan plc = pl;
  void *params[] = {&a, &plc};
  return ls::launch_sequence<T>(s, a, (const void *)gemm_kernel<T>, params,
                                (size_t)pl.total * sizeof(T), stream);
}

GemmPlan make_plan(int LB, int nP, int nxP, int nuP) {
  GemmPlan p;
  p.LB = LB;
  p.LP = (LB + 2) | 1;  // odd: the column-wise stores of the hats hit distinct banks
  p.nP = nP; p.nxP = nxP; p.nuP = nuP;
  auto up = [](int v) { return (v + 7) / 8 * 8; };
  int o = 0;
  p.oG = o; o += up(nxP * nP);
  p.oGT = o; o += up(nP * nxP);
  p.oH = o; o += up(nP * nP);
  p.oM = o; o += up(nuP * nuP);
  p.oB = o; o += up(nxP * nuP);
  p.oE = o; o += up(nxP);
  p.oHAT = o; o += up(5 * nP * p.LP);
  p.oX1 = o; o += up(nP * p.LP);
  p.oX2 = o; o += up(nP * p.LP);
  p.oT = o; o += up(nuP * p.LP);
  p.oDU = o; o += up(nuP * p.LP);
  p.total = o;
  return p;
}

}  // namespace

int gemm_threads() { return kGemmThreads; }

// The stages per block that fit `budget` bytes of shared memory (at most 128), and the plan.
int gemm_plan(int max_n, int max_nx, int max_nu, int precision, size_t budget, int *plan) {
  const int ts = precision == 0 ? 4 : 8;
  const int nP = (max_n + 3) & ~3, nxP = (max_nx + 3) & ~3, nuP = (max_nu + 3) & ~3;
  for (int LB = 128; LB >= 4; --LB) {
    const GemmPlan p = make_plan(LB, nP, nxP, nuP);
    if ((size_t)p.total * ts <= budget) {
      plan[0] = LB; plan[1] = nP; plan[2] = nxP; plan[3] = nuP; plan[4] = p.total * ts;
      return LB;
    }
  }
  return 0;
}

cudaError_t gemm_configure(int precision, size_t smem, int *blocks_per_sm) {
  cudaError_t rc;
  if (precision == 0) {
    rc = cudaFuncSetAttribute(gemm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, gemm_kernel<float>, kGemmThreads, smem);
  }
  rc = cudaFuncSetAttribute(gemm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (rc != cudaSuccess) return rc;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, gemm_kernel<double>, kGemmThreads, smem);
}

cudaError_t launch_gemm(const AdmmLaunch &s, int precision, const int *plan, cudaStream_t stream) {
  const GemmPlan pl = make_plan(plan[0], plan[1], plan[2], plan[3]);
  return precision == 0 ? launch_t<float>(s, pl, stream) : launch_t<double>(s, pl, stream);
}

}  // namespace pimpc

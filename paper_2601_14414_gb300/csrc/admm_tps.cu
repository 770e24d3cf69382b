// admm_tps.cu -- Algorithm 1 with one thread per stage (instances with n = nx + nu <= 32).
//
// Layout. Stage data of a stage-varying instance is stored in tiles of 32 consecutive stages,
// element-major inside a tile: element e of stage k sits at tile(k) * 32 W + e * 32 + (k mod 32)
// (W = nx n + nx + n(n+1)/2 + nu(nu+1)/2 elements: G = [A | B] row-major, e, then H and M packed
// lower row-major). A warp reads element e of 32 consecutive stages as one 128-byte line (FP32),
// so every load is a full coalesced line and each instruction serves 32 stages. Stage-invariant
// instances keep two plain blocks (H_k for k < N-1, and H_{N-1}) that all lanes read in broadcast.
// Iterates use the same tiling: component c of vector b (z, v, theta, beta, lambda) of stage k at
// tile(k) * 160 n + (b n + c) * 32 + (k mod 32).
//
// Work. A CTA has WC compute warps (one stage per thread, S = 32 WC stages per sub-chunk) and
// one helper warp. For a sub-chunk [k0, k1) of an item:
//   phase A (step 1, first half): w = vhat_k - betahat_k, du_k = M_k (B_k^T w_x + w_u); and
//            y_k = zhat_k - vhat_k - ebar_k + lambdahat_k, a_{k-1} = Abar_k^T y_k, handed to the
//            thread of stage k-1 through shared memory. Helper lane 0 does the same a-part for
//            stage k1 (the next sub-chunk's first stage).
//   phase B (step 1, second half): h_k = qbar_k + rho (zhat_k - thetahat_k + a_k),
//            xbar_{k+1} = H_k h_k, handed to the thread of stage k+1. Helper lane 1 recomputes
//            xbar_{k0} from stage k0-1 at the first sub-chunk of an item that starts mid-horizon.
//   phase C (steps 2-4): Abar_k xbar_k and Bbar_k du_k from G_k, the (v, z) projection update,
//            the dual updates, the six squared norms of c; new iterates to the third buffer.
// Matrix products loop over rows at run time and over columns in registers (compile-time NN =
// n rounded up to a multiple of 4, with predicates for the n <= c < NN tail).
#include <math.h>

#include "lockstep.cuh"

namespace pimpc {

namespace {

constexpr int kWC = 4;                 // compute warps per CTA
constexpr int kThreads = 32 * (kWC + 1);
constexpr int kS = 32 * kWC;           // stages per sub-chunk
constexpr int kNC = kS + 3;            // shared-memory columns: stages k0-1 .. k1 and spares

template <typename T>
__device__ __forceinline__ T clampv(T x, T lo, T hi) {
  return x < lo ? lo : (x > hi ? hi : x);
}

// Per-stage views.
template <typename T>
struct StageView {
  const T *M;   // element e at M[e * ms]
  int ms;
  const T *Hb;  // block holding H_k (LTI: block 0 or block 1)
  const T *ic, *ip;  // iterates: element (b, c) at ic[(b n + c) * 32]
  T *in;
};

template <typename T>
__device__ __forceinline__ StageView<T> view(const ls::Args<T> &a, int j, int k, int N, int Wt,
                                             const T *Ic, const T *Ip, T *In, int n) {
  StageView<T> v;
  const T *blk = a.blk + a.L.blk[j];
  if (a.L.lti) {
    v.M = blk;
    v.ms = 1;
    v.Hb = blk + ((k < N - 1) ? 0 : Wt);
  } else {
    v.M = blk + (int64_t)(k >> 5) * 32 * Wt + (k & 31);
    v.ms = 32;
    v.Hb = v.M;
  }
  const int64_t o = (int64_t)(k >> 5) * (160 * n) + (k & 31);
  v.ic = Ic + o;
  v.ip = Ip + o;
  v.in = In + o;
  return v;
}

template <typename T>
__device__ __forceinline__ T hat(const StageView<T> &v, int idx, bool use_prev, T f) {
  T c = v.ic[idx * 32];
  if (use_prev) c += f * (c - v.ip[idx * 32]);
  return c;
}

// Phase A's a-part for one stage: a_{k-1} = Abar_k^T y_k, written to column `col` of A.
template <typename T, int NN>
__device__ __forceinline__ void a_part(const StageView<T> &v, int nx, int n, const T *yloc,
                                       T *A, int col) {
  T acc[NN];
#pragma unroll
  for (int c = 0; c < NN; ++c) acc[c] = (T)0;
  for (int r = 0; r < nx; ++r) {
    const T yr = yloc[r];
    const T *row = v.M + (int64_t)r * n * v.ms;
#pragma unroll
    for (int c = 0; c < NN; ++c)
      if (c < n) acc[c] += row[c * v.ms] * yr;
  }
#pragma unroll
  for (int c = 0; c < NN; ++c)
    if (c < n) A[c * kNC + col] = acc[c] + (c >= nx ? yloc[c] : (T)0);
}

// Phase B for one stage: h = qbar + rho (zhat - thetahat + a), xbar_next = H h -> column `xcol`.
template <typename T, int NN>
__device__ __forceinline__ void p4(const StageView<T> &v, int nx, int nu, int n, bool use_prev,
                                   T f, T rho, const T *qd, const T *rf, bool has_a,
                                   const T *A, int acol, T *X, int xcol, T *hloc) {
  T h[NN], yacc[NN];
  const int oH = nx * n + nx;
#pragma unroll
  for (int c = 0; c < NN; ++c) {
    yacc[c] = (T)0;
    h[c] = (T)0;
    if (c < n) {
      const T zc = hat(v, c, use_prev, f);
      const T tc = hat(v, 2 * n + c, use_prev, f);
      const T ac = has_a ? A[c * kNC + acol] : (T)0;
      h[c] = qd[c] * (rf ? rf[c] : (T)0) + rho * (zc - tc + ac);
      hloc[c] = h[c];
    }
  }
  (void)nu;
  for (int i = 0; i < n; ++i) {
    const T hi = hloc[i];
    const T *row = v.Hb + (int64_t)(oH + i * (i + 1) / 2) * v.ms;
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < NN; ++c) {
      if (c <= i) {
        const T hv = row[c * v.ms];
        s += hv * h[c];
        if (c < i) yacc[c] += hv * hi;
      }
    }
    X[i * kNC + xcol] = s;
  }
#pragma unroll
  for (int c = 0; c < NN; ++c)
    if (c < n) X[c * kNC + xcol] += yacc[c];
}

// Steps 2-4 for one component c of one stage.
template <typename T>
__device__ __forceinline__ void elementwise(const StageView<T> &v, int n, int c, T ax, T bd, T ee,
                                            T xn, T lo, T hi, bool use_prev, T f, T &cacc) {
  const T zh = hat(v, c, use_prev, f), vh = hat(v, n + c, use_prev, f);
  const T thh = hat(v, 2 * n + c, use_prev, f), beh = hat(v, 3 * n + c, use_prev, f);
  const T lah = hat(v, 4 * n + c, use_prev, f);
  const T gam = bd + beh - ax - ee + lah;
  const T w = ((T)2 * (xn + thh + ax + ee - lah) + gam) / (T)3;
  const T z = clampv(w, lo, hi);
  const T vv = (T)0.5 * (z + gam);
  const T th = thh + xn - z;
  const T be = beh + bd - vv;
  const T la = lah + z - ax - vv - ee;
  const T d1 = th - thh, d2 = be - beh, d3 = la - lah, d4 = z - zh, d5 = vv - vh, d6 = d4 - d5;
  cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
  v.in[c * 32] = z;
  v.in[(n + c) * 32] = vv;
  v.in[(2 * n + c) * 32] = th;
  v.in[(3 * n + c) * 32] = be;
  v.in[(4 * n + c) * 32] = la;
}

template <typename T, int NN>
__device__ void run_item(const ls::Args<T> &a, int j, int ka, int kb, int it, T *A, T *X,
                         T &cacc) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
  const int Wt = a.L.W[j];
  const int bse = a.base[j];
  const int64_t ib = a.L.Ni[j];
  const T *Ic = a.it[(bse + it) % 3] + ib;
  const T *Ip = a.it[(bse + it + 2) % 3] + ib;
  T *In = a.it[(bse + it + 1) % 3] + ib;
  const double coefd = *(volatile double *)&a.coef[j];
  const T f = (T)coefd;
  const bool use_prev = coefd != 0.0;
  const T rho = (T)a.rho;
  const T *qd = a.qd + a.L.off_n[j];
  const T *ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
  const int refstride = a.ref_per_stage ? n : 0;
  const T *lo = a.lo + a.L.off_n[j], *hi = a.hi + a.L.off_n[j];
  const int oE = nx * n, oM = nx * n + nx + n * (n + 1) / 2;
  T yloc[NN], wloc[NN], tloc[NN], hloc[NN], duloc[NN];

  for (int k0 = ka; k0 < kb; k0 += kS) {
    const int k1 = min(k0 + kS, kb);
    // ---------------- phase A ----------------
    if (warp < kWC) {
      const int k = k0 + 32 * warp + lane;
      if (k < k1) {
        const StageView<T> v = view(a, j, k, N, Wt, Ic, Ip, In, n);
        for (int c = 0; c < n; ++c) {
          const T zc = hat(v, c, use_prev, f), vc = hat(v, n + c, use_prev, f);
          const T bc = hat(v, 3 * n + c, use_prev, f), lc = hat(v, 4 * n + c, use_prev, f);
          wloc[c] = vc - bc;
          yloc[c] = zc - vc + lc - (c < nx ? v.M[(oE + c) * v.ms] : (T)0);
        }
        // a_{k-1} = G_k^T y_x + (0, y_u), handed to stage k-1 (column (k-1) - k0 + 1)
        a_part<T, NN>(v, nx, n, yloc, A, k - k0);
        // t = B_k^T w_x + w_u (second pass over the B columns of G_k, now in L1)
        {
          T tacc[NN];
#pragma unroll
          for (int c = 0; c < NN; ++c) tacc[c] = (T)0;
          for (int r = 0; r < nx; ++r) {
            const T wr = wloc[r];
            const T *row = v.M + (int64_t)(r * n + nx) * v.ms;
#pragma unroll
            for (int c = 0; c < NN; ++c)
              if (c < nu) tacc[c] += row[c * v.ms] * wr;
          }
#pragma unroll
          for (int c = 0; c < NN; ++c)
            if (c < nu) tloc[c] = tacc[c] + wloc[nx + c];
        }
        // du_k = M_k t (M packed lower row-major)
        for (int i = 0; i < nu; ++i) {
          T s = (T)0;
          for (int jj = 0; jj < nu; ++jj) {
            const int e = i >= jj ? i * (i + 1) / 2 + jj : jj * (jj + 1) / 2 + i;
            s += v.M[(oM + e) * v.ms] * tloc[jj];
          }
          duloc[i] = s;
        }
      }
    } else if (lane == 0 && k1 < N) {
      // next stage (k1): a_{k1-1} = Abar_{k1}^T y_{k1}
      const StageView<T> v = view(a, j, k1, N, Wt, Ic, Ip, In, n);
      for (int c = 0; c < n; ++c) {
        const T zc = hat(v, c, use_prev, f), vc = hat(v, n + c, use_prev, f);
        const T lc = hat(v, 4 * n + c, use_prev, f);
        yloc[c] = zc - vc + lc - (c < nx ? v.M[(oE + c) * v.ms] : (T)0);
      }
      a_part<T, NN>(v, nx, n, yloc, A, k1 - k0);
    } else if (lane == 1 && k0 == ka) {
      if (ka == 0)
        for (int c = 0; c < n; ++c) X[c * kNC + 0] = a.xb0[a.L.off_n[j] + c];
    }
    __syncthreads();
    // ---------------- phase B ----------------
    if (warp < kWC) {
      const int k = k0 + 32 * warp + lane;
      if (k < k1) {
        const StageView<T> v = view(a, j, k, N, Wt, Ic, Ip, In, n);
        const int col = k - k0 + 1;
        p4<T, NN>(v, nx, nu, n, use_prev, f, rho, qd, ref ? ref + (int64_t)k * refstride : nullptr,
                  k + 1 < N, A, col, X, col, hloc);
      }
    } else if (lane == 1 && k0 == ka && ka > 0) {
      // xbar_{ka} = H_{ka-1} h_{ka-1}; a_{ka-1} was written to column 0 in phase A
      const StageView<T> v = view(a, j, ka - 1, N, Wt, Ic, Ip, In, n);
      p4<T, NN>(v, nx, nu, n, use_prev, f, rho, qd,
                ref ? ref + (int64_t)(ka - 1) * refstride : nullptr, true, A, 0, X, 0, hloc);
    }
    __syncthreads();
    // ---------------- phase C ----------------
    if (warp < kWC) {
      const int k = k0 + 32 * warp + lane;
      if (k < k1) {
        const StageView<T> v = view(a, j, k, N, Wt, Ic, Ip, In, n);
        const int col = k - k0;  // xbar_k in column col, xbar_{k+1} in col + 1
        T xk[NN];
#pragma unroll
        for (int c = 0; c < NN; ++c) xk[c] = c < n ? X[c * kNC + col] : (T)0;
        for (int r = 0; r < nx; ++r) {
          const T *row = v.M + (int64_t)r * n * v.ms;
          T s1 = (T)0, s2 = (T)0;
#pragma unroll
          for (int c = 0; c < NN; ++c)
            if (c < n) s1 += row[c * v.ms] * xk[c];
          for (int c = 0; c < nu; ++c) s2 += row[(nx + c) * v.ms] * duloc[c];
          elementwise(v, n, r, s1, s2, v.M[(oE + r) * v.ms], X[r * kNC + col + 1], lo[r], hi[r],
                      use_prev, f, cacc);
        }
        for (int c = nx; c < n; ++c)
          elementwise(v, n, c, X[c * kNC + col], duloc[c - nx], (T)0, X[c * kNC + col + 1], lo[c],
                      hi[c], use_prev, f, cacc);
      }
    }
    __syncthreads();
    // xbar at the end of this sub-chunk is xbar_k of the next one's first stage
    for (int c = tid; c < n; c += blockDim.x) X[c * kNC + 0] = X[c * kNC + (k1 - k0)];
    __syncthreads();
  }
}

template <typename T>
__device__ void dispatch(const ls::Args<T> &a, int j, int ka, int kb, int it, T *A, T *X, T &cacc) {
  const int n = a.L.nx[j] + a.L.nu[j];
  switch ((n + 3) >> 2) {
    case 1: run_item<T, 4>(a, j, ka, kb, it, A, X, cacc); break;
    case 2: run_item<T, 8>(a, j, ka, kb, it, A, X, cacc); break;
    case 3: run_item<T, 12>(a, j, ka, kb, it, A, X, cacc); break;
    case 4: run_item<T, 16>(a, j, ka, kb, it, A, X, cacc); break;
    case 5: run_item<T, 20>(a, j, ka, kb, it, A, X, cacc); break;
    case 6: run_item<T, 24>(a, j, ka, kb, it, A, X, cacc); break;
    case 7: run_item<T, 28>(a, j, ka, kb, it, A, X, cacc); break;
    default: run_item<T, 32>(a, j, ka, kb, it, A, X, cacc); break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 2) tps_kernel(ls::Args<T> a, int nn_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sItem, sOk;
  __shared__ double sRed[kWC + 1];
  T *A = reinterpret_cast<T *>(smem_raw);
  T *X = A + nn_max * kNC;
  const int tid = threadIdx.x;
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;
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
      const int j = a.item_inst[item];
      if (*(volatile int *)&a.stop[j]) continue;
      T cacc = (T)0;
      dispatch<T>(a, j, a.item_a[item], a.item_b[item], it, A, X, cacc);
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if ((tid & 31) == 0) sRed[tid >> 5] = (double)cacc;
      __syncthreads();
      if (tid == 0) {
        double part = 0.0;
        for (int w = 0; w < kWC + 1; ++w) part += sRed[w];
        ls::finish_item(a, j, it, part);
      }
    }
    if (blockIdx.x == 0 && tid == 0) ctl->queue[(it + 1) & 1] = 0;
    if (!ls::grid_sync(ctl, nblocks, &sOk)) break;
    if (*(volatile int *)&ctl->active <= 0) break;
    if (!ls::compact(a, cl, nact, &sOk, reinterpret_cast<int *>(sRed))) break;
  }
}

}  // namespace

int tps_threads() { return kThreads; }
int tps_stages_per_subchunk() { return kS; }

size_t tps_smem_bytes(int nn_max, int precision) {
  return (size_t)2 * nn_max * kNC * (precision == 0 ? 4 : 8);
}

cudaError_t tps_configure(int precision, size_t smem, int *blocks_per_sm) {
  cudaError_t rc;
  if (precision == 0) {
    rc = cudaFuncSetAttribute(tps_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tps_kernel<float>, kThreads, smem);
  }
  rc = cudaFuncSetAttribute(tps_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (rc != cudaSuccess) return rc;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tps_kernel<double>, kThreads, smem);
}

template <typename T>
static cudaError_t tps_launch_t(const AdmmLaunch &s, cudaStream_t stream) {
  ls::Args<T> a = ls::make_args<T>(s);
  int nn_max = s.nv_max;
  void *params[] = {&a, &nn_max};
  const size_t smem = tps_smem_bytes(nn_max, sizeof(T) == 4 ? 0 : 1);
  return ls::launch_sequence<T>(s, a, (const void *)tps_kernel<T>, params, smem, stream);
}

cudaError_t launch_tps(const AdmmLaunch &s, int precision, cudaStream_t stream) {
  return precision == 0 ? tps_launch_t<float>(s, stream) : tps_launch_t<double>(s, stream);
}

}  // namespace pimpc

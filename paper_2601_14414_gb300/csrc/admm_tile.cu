// admm_tile.cu -- Algorithm 1 with one thread per stage on halo tiles: the batched solve of
// stage-varying FP32 instances (n <= 32).
//
// Layout. Each instance is cut into tiles of tw slots (tw = 32 or 16, chosen so that one tile
// fits the CTA's shared memory): tile t holds stages t P - 1 .. t P + P in slots 0 .. tw - 1 with
// P = tw - 2 own stages; slot 0 and slot tw - 1 repeat the neighbours' boundary stages (the
// stage data is stored there by the factorisation, the iterates by this kernel), so one
// iteration on a tile reads nothing outside the tile. Every array of a tile is element-major
// (element e of slot s at e tw + s): lane s of a warp reads consecutive words, and the element
// offsets are compile-time immediates.
//
// Work. One cooperative launch runs all iterations of all instances in lock-step (the frame of
// lockstep.cuh): a CTA of 4 warps pulls items of up to 4 consecutive tiles of one instance, copies
// the stage data and the iterate tiles (current, and previous when the momentum factor is
// nonzero) into shared memory with cp.async.bulk on an mbarrier (one bounded wait), and each
// warp runs the iteration on one tile, lane s on slot s:
//   phase 1a (slots 1 .. tw-1): y_k = zhat_k - vhat_k - ebar_k + lambdahat_k and
//            a_{k-1} = Abar_k^T y_k, handed to lane s-1; own slots also form
//            du_k = M_k (B_k^T t_x + t_u), t = vhat_k - betahat_k (Algorithm 1 step 1);
//   phase 1b (slots 0 .. P): h_k = qbar_k + rho (zhat_k - thetahat_k + a_k) and
//            xbar_{k+1} = H_k h_k, handed to lane s+1 (slot 0 recomputes xbar of the first own
//            stage from the left neighbour's data);
//   phase 2  (own slots): Abar_k xbar_k, Bbar_k du_k, the (v, z) projection update, the dual
//            updates and the six squared norms of c (steps 2-4); the new iterate is stored to
//            the tile in global memory (coalesced: one line per element for 32 slots) and the
//            boundary stages also to the neighbouring tiles' halo slots.
// Matrix products run over runtime rows with the columns unrolled to a compile-time bound NN
// (n rounded up to a multiple of 8) in register arrays; vectors that need runtime indices go
// through a per-warp exchange area in shared memory.
#include <math.h>

#include "bulk.cuh"
#include "lockstep.cuh"

namespace pimpc {

namespace {

using namespace bulk;

template <typename T>
using Args = ls::Args<T>;

constexpr int kTileWarps = 4;
constexpr int kTileThreads = 32 * kTileWarps;

template <typename T>
struct TileJob {
  int n, nx, nu, N, t;
  const T *sB, *sIc, *sIp;  // shared: stage data, current and previous iterate tiles
  T *ex;                     // shared exchange: four rows of n * tw words
  bool use_prev;
  T f, rho;
  const T *qd, *lo, *hi, *xb0;  // per-instance vectors (global)
  const T *ref;                 // reference of stage k at ref + k * ref_stride, or null
  int ref_stride;
  T *In, *InPrev, *InNext;      // new iterate tile t, tiles t-1 / t+1 (null if absent)
};

// sum_{c < cnt} row[c * TW] x[c], cnt <= NN (columns in chunks of four).
template <typename T, int TW, int NN>
__device__ __forceinline__ T dot_row(const T *row, const T (&x)[NN], int cnt) {
  T a0 = (T)0, a1 = (T)0;
#pragma unroll
  for (int c0 = 0; c0 < NN; c0 += 4) {
    if (c0 >= cnt) break;
#pragma unroll
    for (int c = c0; c < c0 + 4; ++c)
      if (c < cnt) {
        if (c & 1) a1 += row[c * TW] * x[c];
        else a0 += row[c * TW] * x[c];
      }
  }
  return a0 + a1;
}

// acc[c] += row[c * TW] s for c < cnt.
template <typename T, int TW, int NN>
__device__ __forceinline__ void axpy_row(const T *row, T s, T (&acc)[NN], int cnt) {
#pragma unroll
  for (int c0 = 0; c0 < NN; c0 += 4) {
    if (c0 >= cnt) break;
#pragma unroll
    for (int c = c0; c < c0 + 4; ++c)
      if (c < cnt) acc[c] += row[c * TW] * s;
  }
}

// out = S x for a symmetric m x m matrix S packed lower row-major (element (i, c), c <= i, at
// S[(i (i + 1) / 2 + c) * TW]); x in registers and in xs[c * TW]; tmp[i * TW] is scratch.
template <typename T, int TW, int NN>
__device__ __forceinline__ void spmv(const T *S, int m, const T (&x)[NN], const T *xs, T *tmp,
                                     T (&out)[NN]) {
#pragma unroll
  for (int c = 0; c < NN; ++c) out[c] = (T)0;
  for (int i = 0; i < m; ++i) {
    const T xi = xs[i * TW];
    const T *row = S + (i * (i + 1) / 2) * TW;
    T acc = (T)0;
#pragma unroll
    for (int c0 = 0; c0 < NN; c0 += 4) {
      if (c0 > i) break;
#pragma unroll
      for (int c = c0; c < c0 + 4; ++c)
        if (c <= i) {
          const T v = row[c * TW];
          acc += v * x[c];
          if (c < i) out[c] += v * xi;
        }
    }
    tmp[i * TW] = acc;
  }
#pragma unroll
  for (int c = 0; c < NN; ++c)
    if (c < m) out[c] += tmp[c * TW];
}

// One iteration of Algorithm 1 on one tile; every lane of the warp calls it. Returns this
// lane's share of the six squared norms of c (own slots only).
template <typename T, int TW, int NN>
__device__ __noinline__ T tile_iteration(const TileJob<T> &J) {
  constexpr int P = TW - 2;
  const int s = threadIdx.x & 31;
  const bool in = s < TW;
  const int n = J.n, nx = J.nx, nu = J.nu, N = J.N;
  const int k = J.t * P - 1 + s;
  const bool valid = in && k >= 0 && k < N;
  const bool own = in && s >= 1 && s <= P && k < N;
  const int nT = n * TW;
  const T *G = J.sB + s;                    // G[r][c] at G[(r n + c) TW]
  const T *Ev = G + nx * nT;                // e[r]
  const T *Hp = Ev + nx * TW;               // H packed lower
  const T *Mp = Hp + (n * (n + 1) / 2) * TW;  // M packed lower
  const T *Ic = J.sIc + s, *Ip = J.sIp + s;
  T *X0 = J.ex + s, *XA = X0 + nT, *XX = XA + nT, *XH = XX + nT;  // exchange rows (column s)
  const bool up = J.use_prev;
  const T f = J.f;
  auto hat = [&](int b, int c) -> T {
    const int o = (b * n + c) * TW;
    T v = Ic[o];
    if (up) v += f * (v - Ip[o]);
    return v;
  };
  T cacc = (T)0;

  // ---- phase 1a ----
  T du[NN];
#pragma unroll
  for (int q = 0; q < NN; ++q) du[q] = (T)0;
  if (in && s >= 1) {
    if (valid) {
      for (int c = 0; c < n; ++c)
        X0[c * TW] = hat(0, c) - hat(1, c) + hat(4, c) - (c < nx ? Ev[c * TW] : (T)0);
      T a[NN];
#pragma unroll
      for (int c = 0; c < NN; ++c) a[c] = (c >= nx && c < n) ? X0[c * TW] : (T)0;
      for (int r = 0; r < nx; ++r) axpy_row<T, TW, NN>(G + r * nT, X0[r * TW], a, n);
#pragma unroll
      for (int c = 0; c < NN; ++c)
        if (c < n) XA[c * TW - 1] = a[c];  // a_{k-1} -> lane s-1
    } else {
      for (int c = 0; c < n; ++c) XA[c * TW - 1] = (T)0;  // stage k = N: none for k-1 = N-1
    }
  }
  if (own) {
    T tv[NN], w[NN];
#pragma unroll
    for (int c = 0; c < NN; ++c) {
      tv[c] = (T)0;
      if (c < n) {
        tv[c] = hat(1, c) - hat(3, c);
        XH[c * TW] = tv[c];
      }
    }
#pragma unroll
    for (int q = 0; q < NN; ++q) w[q] = (T)0;
    for (int r = 0; r < nx; ++r) axpy_row<T, TW, NN>(G + r * nT + nx * TW, XH[r * TW], w, nu);
#pragma unroll
    for (int q = 0; q < NN; ++q)
      if (q < nu) {
        w[q] += XH[(nx + q) * TW];  // w = B_k^T t_x + t_u
        X0[q * TW] = w[q];
      }
    spmv<T, TW, NN>(Mp, nu, w, X0, XX, du);  // du_k = M_k w
  }
  __syncwarp();

  // ---- phase 1b ----
  T xo[NN];
#pragma unroll
  for (int c = 0; c < NN; ++c) xo[c] = (T)0;
  if (valid && s <= P) {
    const T *rf = J.ref ? J.ref + (int64_t)k * J.ref_stride : nullptr;
    T h[NN];
#pragma unroll
    for (int c = 0; c < NN; ++c) {
      h[c] = (T)0;
      if (c < n) {
        h[c] = J.qd[c] * (rf ? rf[c] : (T)0) + J.rho * (hat(0, c) - hat(2, c) + XA[c * TW]);
        XH[c * TW] = h[c];
      }
    }
    spmv<T, TW, NN>(Hp, n, h, XH, X0, xo);  // xbar_{k+1} = H_k h_k
#pragma unroll
    for (int c = 0; c < NN; ++c)
      if (c < n) XX[c * TW + 1] = xo[c];     // -> lane s+1
  } else if (in && s == 0 && k < 0) {
    for (int c = 0; c < n; ++c) XX[c * TW + 1] = J.xb0[c];  // first tile: xbar_0
  }
  __syncwarp();

  // ---- phase 2 ----
  if (own) {
    T xk[NN];
#pragma unroll
    for (int c = 0; c < NN; ++c) xk[c] = c < n ? XX[c * TW] : (T)0;
#pragma unroll
    for (int c = 0; c < NN; ++c)
      if (c < n) XH[c * TW] = xo[c];
#pragma unroll
    for (int q = 0; q < NN; ++q)
      if (q < nu) X0[q * TW] = du[q];
    T *o = J.In + s;
    for (int r = 0; r < n; ++r) {
      T ax, bd, ee;
      if (r < nx) {
        const T *row = G + r * nT;
        ax = dot_row<T, TW, NN>(row, xk, n);
        bd = dot_row<T, TW, NN>(row + nx * TW, du, nu);
        ee = Ev[r * TW];
      } else {
        ax = XX[r * TW];
        bd = X0[(r - nx) * TW];
        ee = (T)0;
      }
      const T zh = hat(0, r), vh = hat(1, r), thh = hat(2, r), beh = hat(3, r), lah = hat(4, r);
      const T xn = XH[r * TW];
      const T gam = bd + beh - ax - ee + lah;
      const T w = ((T)2 * (xn + thh + ax + ee - lah) + gam) / (T)3;
      const T lo = J.lo[r], hi = J.hi[r];
      const T z = w < lo ? lo : (w > hi ? hi : w);
      const T v = (T)0.5 * (z + gam);
      const T th = thh + xn - z;
      const T be = beh + bd - v;
      const T la = lah + z - ax - v - ee;
      const T d1 = th - thh, d2 = be - beh, d3 = la - lah, d4 = z - zh, d5 = v - vh, d6 = d4 - d5;
      cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
      o[r * TW] = z;
      o[(n + r) * TW] = v;
      o[(2 * n + r) * TW] = th;
      o[(3 * n + r) * TW] = be;
      o[(4 * n + r) * TW] = la;
      if (s == P && J.InNext) {  // left halo of tile t+1: z, theta
        J.InNext[r * TW] = z;
        J.InNext[(2 * n + r) * TW] = th;
      }
      if (s == 1 && J.InPrev) {  // right halo of tile t-1: z, v, lambda
        J.InPrev[r * TW + TW - 1] = z;
        J.InPrev[(n + r) * TW + TW - 1] = v;
        J.InPrev[(4 * n + r) * TW + TW - 1] = la;
      }
    }
  }
  return cacc;
}

template <typename T>
__device__ T run_tile(const TileJob<T> &J, int tw) {
  const int nn = (J.n + 7) & ~7;
  if (tw == 32) {
    switch (nn) {
      case 8: return tile_iteration<T, 32, 8>(J);
      case 16: return tile_iteration<T, 32, 16>(J);
      case 24: return tile_iteration<T, 32, 24>(J);
      default: return tile_iteration<T, 32, 32>(J);
    }
  }
  switch (nn) {
    case 8: return tile_iteration<T, 16, 8>(J);
    case 16: return tile_iteration<T, 16, 16>(J);
    case 24: return tile_iteration<T, 16, 24>(J);
    default: return tile_iteration<T, 16, 32>(J);
  }
}

// ---------------------------------------------------------------------------------------------
// The persistent kernel.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTileThreads) tile_kernel(Args<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int sItem, sOk, sArr;
  __shared__ double sRed[kTileWarps];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;

  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par = 0u;
  bool pend = false;

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
      const int t0 = a.item_a[item], nt = a.item_b[item] - t0;
      const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
      const int tw = a.L.tw[j];
      const int TB = a.L.W[j], TI = tile_iter_words(tw, n), EXW = 4 * n * tw;
      const int ntiles = halo_tiles(N, tw);
      const double coefd = *(volatile double *)&a.coef[j];
      const bool use_prev = coefd != 0.0;
      const int bse = a.base[j];
      const int64_t ib = a.L.Ni[j];
      const T *Ic = a.it[(bse + it) % 3] + ib;
      const T *Ip = a.it[(bse + it + 2) % 3] + ib;
      T *In = a.it[(bse + it + 1) % 3] + ib;
      const T *blk = a.blk + a.L.blk[j];
      T *sB = sm, *sIc = sB + nt * TB, *sIp = sIc + nt * TI, *sEx = sIp + nt * TI;

      if (tid == 0) {
        const uint32_t bB = (uint32_t)((size_t)nt * TB * sizeof(T));
        const uint32_t bI = (uint32_t)((size_t)nt * TI * sizeof(T));
        fence_proxy_async();
        mbar_expect_tx(&mbar, bB + bI * (use_prev ? 2u : 1u));
        bulk_load(sB, blk + (int64_t)t0 * TB, bB, &mbar);
        bulk_load(sIc, Ic + (int64_t)t0 * TI, bI, &mbar);
        if (use_prev) bulk_load(sIp, Ip + (int64_t)t0 * TI, bI, &mbar);
        pend = true;
        sArr = mbar_wait(&mbar, par, ctl) ? 1 : 0;
        if (sArr) {
          par ^= 1u;
          pend = false;
        }
      }
      __syncthreads();
      if (!sArr) { ok = false; break; }

      T cacc = (T)0;
      if (warp < nt) {
        const int t = t0 + warp;
        TileJob<T> J;
        J.n = n; J.nx = nx; J.nu = nu; J.N = N; J.t = t;
        J.sB = sB + warp * TB;
        J.sIc = sIc + warp * TI;
        J.sIp = sIp + warp * TI;
        J.ex = sEx + warp * EXW;
        J.use_prev = use_prev;
        J.f = (T)coefd;
        J.rho = (T)a.rho;
        J.qd = a.qd + a.L.off_n[j];
        J.lo = a.lo + a.L.off_n[j];
        J.hi = a.hi + a.L.off_n[j];
        J.xb0 = a.xb0 + a.L.off_n[j];
        J.ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
        J.ref_stride = a.ref_per_stage ? n : 0;
        J.In = In + (int64_t)t * TI;
        J.InPrev = t > 0 ? J.In - TI : nullptr;
        J.InNext = t + 1 < ntiles ? J.In + TI : nullptr;
        cacc = run_tile<T>(J, tw);
      }
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if (lane == 0) sRed[warp] = (double)cacc;
      __syncthreads();
      if (tid == 0) {
        double part = 0.0;
        for (int w = 0; w < kTileWarps; ++w) part += sRed[w];
        a.cpart[item] = part;  // steps 5-7 run in the pass after the barrier
      }
    }
    if (!ok) break;
    if (blockIdx.x == 0 && tid == 0) ctl->queue[(it + 1) & 1] = 0;
    if (!ls::grid_sync(ctl, nblocks, &sOk)) break;
    if (!ls::finish_pass(a, it, cl, nblocks, &sOk)) break;
    if (*(volatile int *)&ctl->active <= 0) break;
    if (!ls::compact(a, cl, nact, &sOk, reinterpret_cast<int *>(sRed))) break;
  }
  // Never leave a bulk copy in flight into shared memory: wait (bounded) for a pending phase.
  if (tid == 0 && pend) {
    long long w = 0;
    while (!mbar_try_wait(&mbar, par) && ++w < ls::kWaitLimit) {
    }
  }
}

}  // namespace

int tile_threads() { return kTileThreads; }
int tile_warps() { return kTileWarps; }

cudaError_t tile_configure(size_t smem, int *blocks_per_sm) {
  cudaError_t rc = cudaFuncSetAttribute(tile_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
  if (rc != cudaSuccess) return rc;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tile_kernel<float>,
                                                       kTileThreads, smem);
}

cudaError_t launch_tile(const AdmmLaunch &s, cudaStream_t stream) {
  Args<float> a = ls::make_args<float>(s);
  void *params[] = {&a};
  return ls::launch_sequence<float>(s, a, (const void *)tile_kernel<float>, params,
                                    (size_t)s.capB * sizeof(float), stream);
}

}  // namespace pimpc

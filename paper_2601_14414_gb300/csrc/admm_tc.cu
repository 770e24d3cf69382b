// admm_tc.cu -- Algorithm 1 on stage-invariant instances with the stage products on the tensor
// cores (schedule family 6, FP32 iterations, iterate layout 4).
//
// With A, B, e shared by every stage, the per-stage products of Algorithm 1 step 1 and step 2
// over a tile of stages are matrix-matrix products with one row per stage:
//   G1  t   = W_x B            (W = vhat - betahat; t + W_u = Bbar^T (vhat - betahat))
//   G2  du  = (t + W_u) M      (M = (B^T B + I + Wdu / rho)^{-1}, symmetric)
//   G3  q   = Y_x [A | B]      (y = zhat - vhat - ebar + lambdahat of the next stage;
//                               Abar^T y = [A^T y_x ; B^T y_x + y_u])
//   G4  xb  = h H              (h = qbar + rho (zhat - thetahat + Abar^T y); H symmetric)
//   G5  ax  = Xbar [A | B]^T   (the x part of Abar xbar_k; its u part is u_k itself)
//   G6  bd  = du B^T           (the x part of Bbar du_k; its u part is du_k)
// and then steps 2-4 elementwise. Each product is D (128 stages x N) = A (128 x K) B^T (N x K) on
// tcgen05.mma of kind::tf32 with the FP32 accumulator in tensor memory; FP32 accuracy comes from
// splitting both operands into TF32 pairs, x = x_hi + x_lo, and adding x_hi y_hi + x_lo y_hi +
// x_hi y_lo (the x_lo y_lo term is below FP32 rounding): three MMAs per K step.
//
// A tile is 128 rows: row 0 is the stage before the tile (its xbar_{k+1} = H h feeds the tile's
// first stage, so it is recomputed here instead of read from a neighbour), rows 1 .. 127 are the
// tile's 127 stages. One CTA (512 threads) per SM; thread t owns row 32 (w % 4) + lane of its
// warp w, which is the tensor-memory lane its warp may read, and the warps w, w + 4, w + 8 and
// w + 12 split the row's components in 16-column chunks. The instance's matrices (hi and lo halves, in the
// canonical K-major core-matrix layout) come to shared memory with one bulk copy per work item
// from a per-instance block that a prepare kernel builds from the FP32 stage cache. Iterates are
// stored in tiles of 128 stages, component-major inside a tile, so that the threads of a warp
// (consecutive stages) read and write consecutive words; they are read with ld.global.cg (L2,
// coherent with the other CTAs' writes before the grid barrier).
#include <math.h>

#include <algorithm>

#include "bulk.cuh"
#include "lockstep.cuh"
#include "tc.cuh"

namespace pimpc {

namespace {

using namespace bulk;
using ls::Args;

constexpr int kRows = 128;         // MMA M: stages per tile plus the halo row
constexpr int kTile = kRows - 1;   // stages a tile updates
constexpr int kThreads = 512;
constexpr int kSplit = kThreads / 128;  // warps sharing a TMEM lane quarter split the columns
constexpr uint32_t kTmemCols = 512;  // 256 accumulator columns, 256 for the row's hats

// Padded sizes (x part and u part each rounded up to 16 columns) and the per-instance matrix
// block: each operand as its TF32 hi half followed by its lo half (rows x K, core-matrix layout).
struct TcDims {
  int nx, nu, n, nxp, nup, np;
  int o1, o2, o3, o4, o5, o6, oE, oHT, words;
};

__host__ __device__ inline TcDims tc_dims(int nx, int nu) {
  TcDims d;
  d.nx = nx; d.nu = nu; d.n = nx + nu;
  d.nxp = (nx + 15) & ~15;
  d.nup = (nu + 15) & ~15;
  d.np = d.nxp + d.nup;
  int o = 0;
  d.o1 = o; o += 2 * d.nup * d.nxp;  // G1: B^T      (nup x nxp)
  d.o2 = o; o += 2 * d.nup * d.nup;  // G2: M        (nup x nup)
  d.o3 = o; o += 2 * d.np * d.nxp;   // G3: [A | B]^T rows (np x nxp)
  d.o4 = o; o += 2 * d.np * d.np;    // G4: H        (np x np)
  d.o5 = o; o += 2 * d.nxp * d.np;   // G5: [A | B]  (nxp x np)
  d.o6 = o; o += 2 * d.nxp * d.nup;  // G6: B        (nxp x nup)
  d.oE = o; o += d.nxp;              // e
  d.oHT = o; o += d.np;              // diagonal of H_{N-1} = (Qbar + rho I)^{-1}
  d.words = (o + 31) & ~31;          // 128-byte multiple (one bulk copy)
  return d;
}

// Component of padded column p (x part first, then u part), or -1 for padding.
__host__ __device__ inline int comp_of(const TcDims &d, int p) {
  if (p < d.nxp) return p < d.nx ? p : -1;
  const int i = p - d.nxp;
  return i < d.nu ? d.nx + i : -1;
}

// Entry (i, j) of a symmetric m x m matrix stored as wrapped diagonals (row d <= m/2 holds
// S[c][(c + d) mod m]).
__device__ inline float sym_at(const float *D, int m, int i, int j) {
  int dd = j - i;
  if (dd < 0) dd += m;
  if (2 * dd <= m) return D[dd * m + i];
  dd = m - dd;
  return D[dd * m + j];
}

// Per-instance matrix block from the FP32 plain stage cache (block 0: G = [A | B], e, H_k, M;
// block 1: H_{N-1}), split into TF32 pairs in the core-matrix layout.
__global__ void tc_prep_kernel(Layout L, const float *blk, float *tcm, const int64_t *tc_off) {
  const int j = blockIdx.x;
  const int nx = L.nx[j], nu = L.nu[j], n = nx + nu;
  const TcDims d = tc_dims(nx, nu);
  const float *b0 = blk + L.blk[j];
  const float *b1 = b0 + L.W[j];
  const int ld = odd_ld(n), oE = nx * ld, oH = oE + nx, oM = oH + wrapped_size(n);
  float *out = tcm + tc_off[j];
  auto put = [&](int base, int R, int K, int r, int k, float v) {
    float hi, lo;
    tc::split_tf32(v, hi, lo);
    out[base + tc::core_off(r, k, K)] = hi;
    out[base + R * K + tc::core_off(r, k, K)] = lo;
  };
  for (int t = threadIdx.x; t < d.nup * d.nxp; t += blockDim.x) {  // B^T
    const int r = t / d.nxp, k = t % d.nxp;
    put(d.o1, d.nup, d.nxp, r, k, (r < nu && k < nx) ? b0[k * ld + nx + r] : 0.0f);
  }
  for (int t = threadIdx.x; t < d.nup * d.nup; t += blockDim.x) {  // M
    const int r = t / d.nup, k = t % d.nup;
    put(d.o2, d.nup, d.nup, r, k, (r < nu && k < nu) ? sym_at(b0 + oM, nu, r, k) : 0.0f);
  }
  for (int t = threadIdx.x; t < d.np * d.nxp; t += blockDim.x) {  // q = G^T y_x
    const int r = t / d.nxp, k = t % d.nxp, c = comp_of(d, r);
    put(d.o3, d.np, d.nxp, r, k, (c >= 0 && k < nx) ? b0[k * ld + c] : 0.0f);
  }
  for (int t = threadIdx.x; t < d.np * d.np; t += blockDim.x) {  // H
    const int r = t / d.np, k = t % d.np, c1 = comp_of(d, r), c2 = comp_of(d, k);
    put(d.o4, d.np, d.np, r, k, (c1 >= 0 && c2 >= 0) ? sym_at(b0 + oH, n, c1, c2) : 0.0f);
  }
  for (int t = threadIdx.x; t < d.nxp * d.np; t += blockDim.x) {  // G
    const int r = t / d.np, k = t % d.np, c = comp_of(d, k);
    put(d.o5, d.nxp, d.np, r, k, (r < nx && c >= 0) ? b0[r * ld + c] : 0.0f);
  }
  for (int t = threadIdx.x; t < d.nxp * d.nup; t += blockDim.x) {  // B
    const int r = t / d.nup, k = t % d.nup;
    put(d.o6, d.nxp, d.nup, r, k, (r < nx && k < nu) ? b0[r * ld + nx + k] : 0.0f);
  }
  for (int t = threadIdx.x; t < d.nxp; t += blockDim.x) out[d.oE + t] = t < nx ? b0[oE + t] : 0.0f;
  for (int t = threadIdx.x; t < d.np; t += blockDim.x) {
    const int c = comp_of(d, t);
    out[d.oHT + t] = c >= 0 ? sym_at(b1 + oH, n, c, c) : 0.0f;
  }
}

// Word offset of the 4 padded components p0 .. p0 + 3 (p0 a multiple of 4) of vector b at stage k
// in layout 4 (np = the padded vector length).
__device__ __forceinline__ int64_t it4(int np, int k, int b, int p0) {
  return (int64_t)(k >> 7) * (128 * 5 * np) + (int64_t)(b * np + p0) * 128 + (k & 127) * 4;
}

__device__ __forceinline__ float4 ldcg4(const float *p) {
  return __ldcg(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ void stcg4(float *p, float4 v) { __stcg(reinterpret_cast<float4 *>(p), v); }
__device__ __forceinline__ float &at(float4 &v, int i) { return reinterpret_cast<float *>(&v)[i]; }
__device__ __forceinline__ float at(const float4 &v, int i) {
  return reinterpret_cast<const float *>(&v)[i];
}

struct Bars {
  uint64_t m;        // matrix copy
  uint64_t g[6];     // commits of G1 .. G6
};

__global__ void __launch_bounds__(kThreads, 1) tc_kernel(Args<float> a, const float *tcm,
                                                         const int64_t *tc_off) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) Bars bars;
  __shared__ uint32_t tmem_base;
  __shared__ int sItem, sOk, sInst, sFail;
  __shared__ double sRed[kThreads / 32];
  float *sm = reinterpret_cast<float *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;  // half: this warp's column share (0 .. kSplit-1)
  const int r = 32 * quarter + lane;  // this thread's MMA row / TMEM lane
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;

  if (tid == 0) {
    mbar_init(&bars.m, 1);
    for (int i = 0; i < 6; ++i) mbar_init(&bars.g[i], 1);
    fence_mbar_init();
    sInst = -1;
    sFail = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
  uint32_t parM = 0u, parG = 0u;  // parity bit i: barrier g[i]
  unsigned outstanding = 0u;      // thread 0: commits issued and not yet waited on
  bool mpend = false;
  bool ok = true;

  int cl = 0;
  for (int it = 0; it < a.max_iters && ok; ++it) {
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
      const int ka = a.item_a[item], kb = a.item_b[item];
      const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
      const TcDims d = tc_dims(nx, nu);
      const int np = d.np, nxp = d.nxp, nup = d.nup;
      const int bse = a.base[j];
      const int64_t ib = a.L.Ni[j];
      const float *Ic = a.it[(bse + it) % 3] + ib;
      const float *Ip = a.it[(bse + it + 2) % 3] + ib;
      float *In = a.it[(bse + it + 1) % 3] + ib;
      const double coefd = *(volatile double *)&a.coef[j];
      const float f = (float)coefd;
      const bool use_prev = coefd != 0.0;
      const float rho = (float)a.rho;
      const float *qd = a.qd + a.L.off_n[j];
      const float *ref = a.ref ? (a.ref + (a.ref_per_stage ? a.L.Nn[j] : a.L.off_n[j])) : nullptr;
      const int refstride = a.ref_per_stage ? n : 0;
      const float *lo = a.lo + a.L.off_n[j], *hi = a.hi + a.L.off_n[j];
      const float *xb0 = a.xb0 + a.L.off_n[j];

      float *mat = sm;
      float *bufA = sm + d.words;
      float *bufB = bufA + 2 * kRows * np;
      float *sHTh = bufB + 2 * kRows * np;  // h of the terminal stage (np)
      const int lohalf = kRows * np;        // offset of an A buffer's lo half

      // The instance's matrices (the previous tile's MMAs have all completed).
      if (sInst != j) {
        if (tid == 0) {
          fence_proxy_async();
          mbar_expect_tx(&bars.m, (uint32_t)(d.words * 4));
          bulk_load(mat, tcm + tc_off[j], (uint32_t)(d.words * 4), &bars.m);
        }
        mpend = true;
        const bool arrived = mbar_wait(&bars.m, parM, ctl);
        if (!__syncthreads_and(arrived)) { ok = false; break; }
        parM ^= 1u;
        mpend = false;
        if (tid == 0) sInst = j;
      }
      const float *E = mat + d.oE;
      const float *HT = mat + d.oHT;
      const uint32_t sA = tc::smem_u32(bufA), sB = tc::smem_u32(bufB), sMat = tc::smem_u32(mat);

      // hats of vector b, padded components p0 .. p0 + 3, stage k: cur + f (cur - prev)
      // (Algorithm 1 steps 6-7); one 16-byte load per buffer.
      auto hat4 = [&](int b, int k, int p0) -> float4 {
        const int64_t x = it4(np, k, b, p0);
        float4 cu = ldcg4(Ic + x);
        if (use_prev) {
          const float4 pv = ldcg4(Ip + x);
          cu.x += f * (cu.x - pv.x); cu.y += f * (cu.y - pv.y);
          cu.z += f * (cu.z - pv.z); cu.w += f * (cu.w - pv.w);
        }
        return cu;
      };
      // four consecutive padded columns p0 .. p0 + 3 of one row: one 16-byte store per half
      auto putA4 = [&](float *buf, int row, int p0, float4 v) {
        float4 h, l;
        tc::split_tf32(v.x, h.x, l.x); tc::split_tf32(v.y, h.y, l.y);
        tc::split_tf32(v.z, h.z, l.z); tc::split_tf32(v.w, h.w, l.w);
        const int o = tc::core_off(row, p0, np);
        *reinterpret_cast<float4 *>(buf + o) = h;
        *reinterpret_cast<float4 *>(buf + lohalf + o) = l;
      };
      auto getA4 = [&](const float *buf, int row, int p0) -> float4 {
        const int o = tc::core_off(row, p0, np);
        const float4 h = *reinterpret_cast<const float4 *>(buf + o);
        const float4 l = *reinterpret_cast<const float4 *>(buf + lohalf + o);
        return make_float4(h.x + l.x, h.y + l.y, h.z + l.z, h.w + l.w);
      };
      // D[tcol] = A[:, ak0 .. ak0 + K) x Mat^T, Mat (nrows x K) at word offset moff of the block.
      auto gemm = [&](uint32_t tcol, uint32_t abuf, int ak0, int K, int moff, int nrows) {
        const uint32_t idesc = tc::idesc_tf32(kRows, nrows);
        const uint32_t sboA = (uint32_t)np * 32u, sboB = (uint32_t)K * 32u;
        const uint32_t aHi = abuf + (uint32_t)(ak0 / 4) * 128u, aLo = aHi + (uint32_t)lohalf * 4u;
        const uint32_t bHi = sMat + (uint32_t)moff * 4u, bLo = bHi + (uint32_t)(nrows * K) * 4u;
        for (int s = 0; s < K / 8; ++s) {
          const uint32_t ko = (uint32_t)s * 256u;
          tc::mma_tf32(tcol, tc::smem_desc(aHi + ko, 128u, sboA), tc::smem_desc(bHi + ko, 128u, sboB),
                       idesc, s > 0 ? 1u : 0u);
          tc::mma_tf32(tcol, tc::smem_desc(aLo + ko, 128u, sboA), tc::smem_desc(bHi + ko, 128u, sboB),
                       idesc, 1u);
          tc::mma_tf32(tcol, tc::smem_desc(aHi + ko, 128u, sboA), tc::smem_desc(bLo + ko, 128u, sboB),
                       idesc, 1u);
        }
      };
      // Barrier between the threads' shared-memory writes and the MMAs that read them.
      auto publish = [&]() {
        tc::fence_smem_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
      };
      // A wait that gives up marks the item failed; the threads still pass every barrier of the
      // tile together and leave at its end.
      auto wait_g = [&](int i) {
        const bool arrived = mbar_wait(&bars.g[i], (parG >> i) & 1u, ctl);
        if (arrived) {
          parG ^= (1u << i);
          if (tid == 0) outstanding &= ~(1u << i);
        } else {
          sFail = 1;
        }
        tc::fence_after_sync();
      };
      auto commit = [&](int i) {
        tc::mma_commit(&bars.g[i]);
        outstanding |= (1u << i);
      };
      const uint32_t cT = 0, cDU = (uint32_t)nup, cQ = 2u * nup, cXB = cQ + (uint32_t)np;
      const uint32_t cAX = cXB + (uint32_t)np, cBD = cAX + (uint32_t)nxp;
      // The row's hats zhat, vhat, betahat, lambdahat (loaded in phase A) kept in tensor memory
      // columns 256 + b np + p for phases B and D (thetahat is read where it is used).
      auto cHat = [&](int b) -> uint32_t { return 256u + (uint32_t)(b * np); };
      const int nch = np / 16, nchx = nxp / 16;
      // padded columns that hold no component (x part beyond nx, u part beyond nu) stay zero
      auto valid4 = [&](int p0, int i) -> bool {
        const int p = p0 + i;
        return p < nxp ? p < nx : p - nxp < nu;
      };
      float cacc = 0.0f;

      // L2 prefetch of the 128-stage storage tiles (current and previous iterates) that the
      // compute tile starting at stage kk reads: their HBM reads overlap the work before them.
      const int64_t stile = (int64_t)128 * 5 * np;  // words of one storage tile
      const int ntile_st = (N + 127) >> 7;
      auto prefetch = [&](int kk) {
        const int t0 = max(kk - 1, 0) >> 7, t1 = min(kk + kTile, N - 1) >> 7;
        for (int t = t0; t <= t1 && t < ntile_st; ++t) {
          bulk_prefetch_l2(Ic + t * stile, (uint32_t)(stile * 4));
          if (use_prev) bulk_prefetch_l2(Ip + t * stile, (uint32_t)(stile * 4));
        }
      };
      if (tid == 0) prefetch(ka);
      for (int k0 = ka; k0 < kb; k0 += kTile) {
        const int cnt = min(kTile, kb - k0);
        if (tid == 0 && k0 + kTile < kb) prefetch(k0 + kTile);
        const int k = k0 - 1 + r;
        const bool inb = k >= 0 && k < N;
        const bool own = r >= 1 && r <= cnt;  // rows updated by this tile (all in range)
        const bool term = k == N - 1;
        const bool last = r == kRows - 1 && k + 1 < N;  // the last row also needs stage k + 1

        // ---- phase A: W = vhat - betahat (x part) and y (of the next stage, one row up) ----
        for (int qc = half; qc < nch; qc += kSplit) {
          const bool xq = qc < nchx;
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const int p0 = 16 * qc + 4 * q4;
            float4 y4 = make_float4(0.f, 0.f, 0.f, 0.f), w4 = y4, yn4 = y4;
            float4 z4 = y4, v4 = y4, l4 = y4, b4 = y4;
            if (inb) {
              z4 = hat4(0, k, p0); v4 = hat4(1, k, p0); l4 = hat4(4, k, p0); b4 = hat4(3, k, p0);
              y4 = make_float4(z4.x - v4.x + l4.x, z4.y - v4.y + l4.y, z4.z - v4.z + l4.z,
                               z4.w - v4.w + l4.w);
              if (xq) {
                const float4 e4 = *reinterpret_cast<const float4 *>(E + p0);
                w4 = make_float4(v4.x - b4.x, v4.y - b4.y, v4.z - b4.z, v4.w - b4.w);
                y4.x -= e4.x; y4.y -= e4.y; y4.z -= e4.z; y4.w -= e4.w;
              }
            }
            tc::tmem_st4(trow + cHat(0) + p0, z4);
            tc::tmem_st4(trow + cHat(1) + p0, v4);
            tc::tmem_st4(trow + cHat(2) + p0, b4);
            tc::tmem_st4(trow + cHat(3) + p0, l4);
            if (last) {
              const float4 z4 = hat4(0, k + 1, p0), v4 = hat4(1, k + 1, p0), l4 = hat4(4, k + 1, p0);
              yn4 = make_float4(z4.x - v4.x + l4.x, z4.y - v4.y + l4.y, z4.z - v4.z + l4.z,
                                z4.w - v4.w + l4.w);
              if (xq) {
                const float4 e4 = *reinterpret_cast<const float4 *>(E + p0);
                yn4.x -= e4.x; yn4.y -= e4.y; yn4.z -= e4.z; yn4.w -= e4.w;
              }
            }
            if (xq) {
              putA4(bufA, r, p0, w4);
              if (r >= 1) putA4(bufB, r - 1, p0, y4);
              if (r == kRows - 1) putA4(bufB, r, p0, yn4);
            } else {  // y_u: not an MMA operand, read back in phase B
              if (r >= 1) *reinterpret_cast<float4 *>(bufB + tc::core_off(r - 1, p0, np)) = y4;
              if (r == kRows - 1) *reinterpret_cast<float4 *>(bufB + tc::core_off(r, p0, np)) = yn4;
            }
          }
        }
        tc::tmem_wait_st();
        publish();
        if (tid == 0) {
          gemm(cT, sA, 0, nxp, d.o1, nup);
          commit(0);
          gemm(cQ, sB, 0, nxp, d.o3, np);
          commit(1);
        }

        // ---- phase B: t + W_u (input of G2), then h (input of G4, in bufA once G2 is done) ----
        wait_g(0);
        for (int qc = nchx + half; qc < nch; qc += kSplit) {
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const int p0 = 16 * qc + 4 * q4;
            const float4 t4 = tc::tmem_ld4(trow + cT + (p0 - nxp));
            const float4 v4 = tc::tmem_ld4(trow + cHat(1) + p0), b4 = tc::tmem_ld4(trow + cHat(2) + p0);
            float4 v2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (inb) {
              v2 = make_float4(t4.x + v4.x - b4.x, t4.y + v4.y - b4.y, t4.z + v4.z - b4.z,
                               t4.w + v4.w - b4.w);
            }
            putA4(bufA, r, p0, v2);  // bufA columns nxp .. np: the G2 operand
          }
        }
        publish();
        if (tid == 0) {
          gemm(cDU, sA, nxp, nup, d.o2, nup);
          commit(2);
        }
        wait_g(1);
        wait_g(2);  // G2 has read bufA: h may overwrite it
        for (int qc = half; qc < nch; qc += kSplit) {
          const bool xq = qc < nchx;
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const int p0 = 16 * qc + 4 * q4;
            const float4 q4v = tc::tmem_ld4(trow + cQ + p0);
            const float4 z4 = tc::tmem_ld4(trow + cHat(0) + p0);
            float4 h4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (inb) {
              const float4 t4 = hat4(2, k, p0);
              // y_u of this row (the row below wrote it in phase A)
              const float4 yu4 = xq ? make_float4(0.f, 0.f, 0.f, 0.f)
                                    : *reinterpret_cast<const float4 *>(bufB + tc::core_off(r, p0, np));
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int p = p0 + i;
                if (!valid4(p0, i)) continue;
                const int c = p < nxp ? p : nx + (p - nxp);
                const float rf = ref ? qd[c] * __ldg(ref + (int64_t)k * refstride + c) : 0.0f;
                at(h4, i) = rf + rho * (at(z4, i) - at(t4, i) + at(q4v, i) + at(yu4, i));
              }
            }
            putA4(bufA, r, p0, h4);
            if (term) *reinterpret_cast<float4 *>(sHTh + p0) = h4;
          }
        }
        publish();
        if (tid == 0) {
          gemm(cXB, sA, 0, np, d.o4, np);
          commit(3);
        }

        // ---- phase C: du (input of G6, bufB columns 0 .. nup), then xbar shifted one row down
        // (input of G5, in bufA once G4 is done) ----
        for (int qc = nchx + half; qc < nch; qc += kSplit) {
          const int su = qc - nchx;  // u chunk: du columns 16 su .. 16 su + 15
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const float4 du4 = tc::tmem_ld4(trow + cDU + 16 * su + 4 * q4);
            putA4(bufB, r, 16 * su + 4 * q4, inb ? du4 : make_float4(0.f, 0.f, 0.f, 0.f));
          }
        }
        publish();
        if (tid == 0) {
          gemm(cBD, sB, 0, nup, d.o6, nxp);
          commit(4);
        }
        wait_g(3);
        for (int qc = half; qc < nch; qc += kSplit) {
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const int p0 = 16 * qc + 4 * q4;
            const float4 xb = tc::tmem_ld4(trow + cXB + p0);
            if (r + 1 < kRows) {
              float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
              if (k < 0) {  // stage 0 starts from xbar_0
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const int p = p0 + i;
                  if (valid4(p0, i)) at(v4, i) = xb0[p < nxp ? p : nx + (p - nxp)];
                }
              } else if (inb) {
                if (term) {
                  const float4 hh = *reinterpret_cast<const float4 *>(sHTh + p0);
                  const float4 ht = *reinterpret_cast<const float4 *>(HT + p0);
                  v4 = make_float4(ht.x * hh.x, ht.y * hh.y, ht.z * hh.z, ht.w * hh.w);
                } else {
                  v4 = xb;
                }
              }
              putA4(bufA, r + 1, p0, v4);
            }
            if (r == 0) putA4(bufA, 0, p0, make_float4(0.f, 0.f, 0.f, 0.f));  // never used
          }
        }
        publish();
        if (tid == 0) {
          gemm(cAX, sA, 0, np, d.o5, nxp);
          commit(5);
        }

        // ---- phase D: steps 2-4 on the tile's stages ----
        wait_g(4);
        wait_g(5);
        for (int qc = half; qc < nch; qc += kSplit) {
          const bool xq = qc < nchx;
#pragma unroll 2
          for (int q4 = 0; q4 < 4; ++q4) {
            const int p0 = 16 * qc + 4 * q4;
            // Abar xbar_k and Bbar du_k: x part from G5 / G6, u part u_{k-1} (bufA) and du_k
            const float4 ax4 = xq ? tc::tmem_ld4(trow + cAX + p0) : getA4(bufA, r, p0);
            const float4 bd4 = xq ? tc::tmem_ld4(trow + cBD + p0) : tc::tmem_ld4(trow + cDU + (p0 - nxp));
            float4 xn4 = tc::tmem_ld4(trow + cXB + p0);
            const float4 z4 = tc::tmem_ld4(trow + cHat(0) + p0), v4 = tc::tmem_ld4(trow + cHat(1) + p0);
            const float4 b4 = tc::tmem_ld4(trow + cHat(2) + p0), l4 = tc::tmem_ld4(trow + cHat(3) + p0);
            if (!own) continue;
            const float4 t4 = hat4(2, k, p0);
            const float4 e4 = xq ? *reinterpret_cast<const float4 *>(E + p0) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (term) {
              const float4 hh = *reinterpret_cast<const float4 *>(sHTh + p0);
              const float4 ht = *reinterpret_cast<const float4 *>(HT + p0);
              xn4 = make_float4(ht.x * hh.x, ht.y * hh.y, ht.z * hh.z, ht.w * hh.w);
            }
            float4 oz, ov, ot, ob, ol;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int p = p0 + i;
              if (!valid4(p0, i)) {
                at(oz, i) = at(ov, i) = at(ot, i) = at(ob, i) = at(ol, i) = 0.0f;
                continue;
              }
              const int c = p < nxp ? p : nx + (p - nxp);
              const float ax = at(ax4, i), bd = at(bd4, i), ee = at(e4, i), xn = at(xn4, i);
              const float zh = at(z4, i), vh = at(v4, i), th = at(t4, i), bh = at(b4, i), lh = at(l4, i);
              const float gam = bd + bh - ax - ee + lh;
              const float w = (2.0f * (xn + th + ax + ee - lh) + gam) / 3.0f;
              const float z = fminf(fmaxf(w, lo[c]), hi[c]);
              const float v = 0.5f * (z + gam);
              const float tt = th + xn - z;
              const float be = bh + bd - v;
              const float lam = lh + z - ax - v - ee;
              const float d1 = tt - th, d2 = be - bh, d3 = lam - lh;
              const float d4 = z - zh, d5 = v - vh, d6 = d4 - d5;
              cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
              at(oz, i) = z; at(ov, i) = v; at(ot, i) = tt; at(ob, i) = be; at(ol, i) = lam;
            }
            stcg4(In + it4(np, k, 0, p0), oz);
            stcg4(In + it4(np, k, 1, p0), ov);
            stcg4(In + it4(np, k, 2, p0), ot);
            stcg4(In + it4(np, k, 3, p0), ob);
            stcg4(In + it4(np, k, 4, p0), ol);
          }
        }
        tc::fence_before_sync();
        __syncthreads();  // bufA / bufB are rewritten by the next tile
        tc::fence_after_sync();
        if (*(volatile int *)&sFail) break;  // uniform: read after the barrier
      }
      if (*(volatile int *)&sFail) { ok = false; break; }

      // ---- step 4: this item's share of c (steps 5-7 follow in the pass after the barrier) ----
      for (int off = 16; off > 0; off >>= 1) cacc += __shfl_xor_sync(0xffffffffu, cacc, off);
      if (lane == 0) sRed[warp] = (double)cacc;
      __syncthreads();
      if (tid == 0) {
        double part = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) part += sRed[w];
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
  if (!ok && tid == 0) atomicExch(&ctl->err, 3);
  // Never leave with a copy or an MMA in flight: wait (bounded) for what is still pending.
  if (tid == 0) {
    for (int i = 0; i < 6; ++i)
      if (outstanding & (1u << i)) {
        long long w = 0;
        while (!mbar_try_wait(&bars.g[i], (parG >> i) & 1u) && ++w < ls::kWaitLimit) {
        }
      }
    if (mpend) {
      long long w = 0;
      while (!mbar_try_wait(&bars.m, parM) && ++w < ls::kWaitLimit) {
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

int tc_threads() { return kThreads; }

bool tc_fits(int nx, int nu) {
  const TcDims d = tc_dims(nx, nu);
  return d.np <= 64 && d.nup <= d.nxp;
}

int64_t tc_block_words(int nx, int nu) { return tc_dims(nx, nu).words; }

size_t tc_smem_bytes(int nx, int nu) {
  const TcDims d = tc_dims(nx, nu);
  return (size_t)(d.words + 4 * kRows * d.np + d.np) * sizeof(float);
}

cudaError_t tc_configure(size_t smem, int *blocks_per_sm) {
  cudaError_t rc = cudaFuncSetAttribute(tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (rc != cudaSuccess) return rc;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, tc_kernel, kThreads, smem);
}

cudaError_t launch_tc(const AdmmLaunch &s, const float *tcm, const int64_t *tc_off, size_t smem,
                      cudaStream_t stream) {
  tc_prep_kernel<<<s.L.batch, 256, 0, stream>>>(s.L, (const float *)s.blk, (float *)tcm, tc_off);
  cudaError_t rc = cudaGetLastError();
  if (rc != cudaSuccess) return rc;
  ls::Args<float> a = ls::make_args<float>(s);
  void *params[] = {&a, (void *)&tcm, (void *)&tc_off};
  return ls::launch_sequence<float>(s, a, (const void *)tc_kernel, params, smem, stream);
}

}  // namespace pimpc

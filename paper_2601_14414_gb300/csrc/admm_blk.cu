// admm_blk.cu -- Algorithm 1 with lanes that own 4-column blocks, on blocked stage blocks
// (schedule family 5, tiled layout 3).
//
// The frame is the lock-step persistent one of admm.cu (items of consecutive stages pulled from
// a queue, a grid barrier per iteration, steps 5-7 in the pass over the instances after it, stopped
// instances compacted away). What differs is how a stage's products map onto lanes.
//
// A group of g = 4, 8 or 16 lanes (n <= 16, 32, 64) handles one stage; lane l owns the
// components 4l .. 4l+3 of every stage vector and reads and writes them as 16-byte vectors. The
// products of Algorithm 1 become, per lane, dense 4-wide work:
//   * q_k = Abar_k^T y_k and t_k = B_k^T w_x + w_u (y = zhat - vhat + lambdahat - ebar,
//     w = vhat - betahat, both of stage k) in one pass over the rows of G_k: lane l reads row r's
//     block l and accumulates both. q_k enters h_{k-1}, so the group of stage k-1 reads it;
//   * du_k = M_k t_k (M as scalar wrapped diagonals, one lane per input);
//   * xbar_{k+1} = H_k h_k with H_k stored as wrapped 4 x 4 block diagonals: lane l owns block
//     row l and, per block diagonal d, applies block (l, l+d) and the transpose of block
//     (l-d, l), so every lane runs the same code and every read is a 16-byte vector (the
//     symmetric diagonal blocks are stored as upper triangles, read as 8-byte pairs; the middle
//     diagonal of an even block count is stored once: half the lanes transpose it in registers);
//   * Abar_k xbar_k and B_k du_k by rows (lane l owns rows l, l+g, ...).
// A sub-chunk holds S - 1 stages and the next stage, whose group only forms q (the first stage
// of the next sub-chunk is formed again there). The group left over in the xbar phase of an
// item's first sub-chunk recomputes xbar_a = H_{a-1} h_{a-1} from the halo (the hats of stage
// a-1 and H_{a-1}; q_a comes from the group of stage a).
//
// Data movement as in admm.cu: one cp.async.bulk batch per sub-chunk completing on an mbarrier
// (stage blocks, the next stage's G and e, current and previous iterates, the halo); every wait
// is bounded. While a sub-chunk computes, the next one of the item is prefetched into L2
// (cp.async.bulk.prefetch.L2), so that its copies, issued once the single buffer is free, read
// L2 rather than HBM. The number of groups S of an instance is fixed on the host so that the
// sub-chunk's shared memory fits the budget of the requested CTAs per SM.
#include <math.h>

#include <algorithm>

#include "bulk.cuh"
#include "usets.cuh"
#include "lockstep.cuh"
#include "products.cuh"

namespace pimpc {

namespace {

using ls::kWaitLimit;
using namespace bulk;

template <typename T>
using Args = ls::Args<T>;

constexpr int kThreads = 128;

template <typename T>
struct V4 {
  T v[4];
};

__device__ __forceinline__ V4<float> ld4(const float *p) {
  const float4 q = *reinterpret_cast<const float4 *>(p);
  return {{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ V4<double> ld4(const double *p) {
  const double2 q0 = *reinterpret_cast<const double2 *>(p);
  const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
  return {{q0.x, q0.y, q1.x, q1.y}};
}
__device__ __forceinline__ void st4(float *p, const V4<float> &x) {
  *reinterpret_cast<float4 *>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
__device__ __forceinline__ void st4(double *p, const V4<double> &x) {
  *reinterpret_cast<double2 *>(p) = make_double2(x.v[0], x.v[1]);
  *reinterpret_cast<double2 *>(p + 2) = make_double2(x.v[2], x.v[3]);
}
// Four components of an iterate in global memory, written by other CTAs before the grid
// barrier (read through L2).
__device__ __forceinline__ V4<float> ldg4(const float *p) {
  const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
  return {{q.x, q.y, q.z, q.w}};
}
__device__ __forceinline__ V4<double> ldg4(const double *p) {
  const double2 q0 = __ldcg(reinterpret_cast<const double2 *>(p));
  const double2 q1 = __ldcg(reinterpret_cast<const double2 *>(p + 2));
  return {{q0.x, q0.y, q1.x, q1.y}};
}
// Two consecutive values at an 8-byte (FP32) or 16-byte (FP64) aligned address.
__device__ __forceinline__ void ld2(const float *p, float &x, float &y) {
  const float2 q = *reinterpret_cast<const float2 *>(p);
  x = q.x;
  y = q.y;
}
__device__ __forceinline__ void ld2(const double *p, double &x, double &y) {
  const double2 q = *reinterpret_cast<const double2 *>(p);
  x = q.x;
  y = q.y;
}
template <typename T>
__device__ __forceinline__ V4<T> zero4() {
  return {{(T)0, (T)0, (T)0, (T)0}};
}

// Shared-memory regions of a sub-chunk with S groups (elements of T): LTV stage blocks (S - 1
// blocks and the next stage's G and e), the halo block (H_{a-1}, or both blocks of a
// stage-invariant instance), per-group scratch (5 vectors), the xbar rows (double-buffered, S
// rows each) and the instance's Qbar diagonal and bounds. The iterates do not pass through
// shared memory: each lane reads its own 16-byte pieces of them from L2, where the previous
// sub-chunk prefetched them.
struct Regions {
  int haloB, scr, X, prm, total;
};

__host__ __device__ inline Regions regions(int nx, int nu, int lti, int tsize, int S) {
  const int n = nx + nu, nP = bl_pad4(n);
  const int W = bl_block_words(nx, nu, tsize), ge = bl_oH(nx, nu, tsize);
  Regions r;
  r.haloB = lti ? 0 : bl_pad4((S - 1) * W + ge);
  r.scr = r.haloB + bl_pad4(lti ? 2 * W : bl_sym_words(n));
  r.X = r.scr + S * 5 * nP;
  r.prm = r.X + 2 * S * nP;  // the instance's Qbar diagonal and bounds (3 vectors)
  r.total = r.prm + 3 * nP;
  return r;
}

// (S h) restricted to the rows 4 I .. 4 I + 3, S symmetric in wrapped 4 x 4 block diagonals at
// Hb (nb blocks per row: the diagonal blocks' upper triangles, Df - 1 further full block
// diagonals, then for an even nb the middle one, stored for block rows below nb/2 only), h in
// shared memory (4 nb values).
template <typename T>
__device__ __forceinline__ V4<T> sym_blocks(const T *Hb, const T *h, int nb, int I) {
  V4<T> acc;
  {  // block (I, I) from its upper triangle (five aligned pairs)
    const T *p = Hb + 10 * I;
    T s[10];
#pragma unroll
    for (int q = 0; q < 5; ++q) ld2(p + 2 * q, s[2 * q], s[2 * q + 1]);
    const V4<T> hv = ld4(h + 4 * I);
    acc.v[0] = s[0] * hv.v[0] + s[1] * hv.v[1] + s[2] * hv.v[2] + s[3] * hv.v[3];
    acc.v[1] = s[1] * hv.v[0] + s[4] * hv.v[1] + s[5] * hv.v[2] + s[6] * hv.v[3];
    acc.v[2] = s[2] * hv.v[0] + s[5] * hv.v[1] + s[7] * hv.v[2] + s[8] * hv.v[3];
    acc.v[3] = s[3] * hv.v[0] + s[6] * hv.v[1] + s[8] * hv.v[2] + s[9] * hv.v[3];
  }
  const int Df = bl_full_diags(nb);
  const T *Hf = Hb + bl_diag_words(nb);
  const int rs = (Df - 1) * nb * 4;  // distance between the planes of rows a and a + 1
  int Jp = I, Jm = I;
  for (int d = 1; d < Df; ++d) {
    Jp = (Jp + 1 == nb) ? 0 : Jp + 1;
    Jm = (Jm == 0) ? nb - 1 : Jm - 1;
    const T *bd = Hf + (d - 1) * nb * 4;
    {  // block (I, I + d): rows of the block against h_{I+d}
      const V4<T> hv = ld4(h + 4 * Jp);
      const T *bp = bd + I * 4;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const V4<T> row = ld4(bp + a * rs);
        acc.v[a] += row.v[0] * hv.v[0] + row.v[1] * hv.v[1] + row.v[2] * hv.v[2] + row.v[3] * hv.v[3];
      }
    }
    {  // block (I, I - d) = transpose of block (I - d, I)
      const V4<T> hm = ld4(h + 4 * Jm);
      const T *bm = bd + Jm * 4;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const V4<T> row = ld4(bm + a * rs);
#pragma unroll
        for (int b = 0; b < 4; ++b) acc.v[b] += row.v[b] * hm.v[a];
      }
    }
  }
  if (!(nb & 1)) {
    // The middle diagonal: block (I, I + nb/2) for I < nb/2, else the transpose of block
    // (I - nb/2, I). Both read the same four rows of the stored block; the transposed case swaps
    // the loaded rows' off-diagonal entries (selects, no divergent branch).
    const int hb = nb >> 1;
    const bool up = I < hb;
    const int Is = up ? I : I - hb;
    const V4<T> hv = ld4(h + 4 * (up ? I + hb : Is));
    const T *bp = Hf + rs * 4 + Is * 4;
    V4<T> r[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) r[a] = ld4(bp + a * hb * 4);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a + 1; b < 4; ++b) {
        const T x = r[a].v[b], y = r[b].v[a];
        r[a].v[b] = up ? x : y;
        r[b].v[a] = up ? y : x;
      }
#pragma unroll
    for (int a = 0; a < 4; ++a)
      acc.v[a] += r[a].v[0] * hv.v[0] + r[a].v[1] * hv.v[1] + r[a].v[2] * hv.v[2] + r[a].v[3] * hv.v[3];
  }
  return acc;
}

// Abar xbar and B du of the rows r = l, l + g, ... < nx of G (stride ldg) with the block count a
// compile-time constant; x and du (4 NB values, du zero outside the input blocks from jx on) in
// shared memory. Row r's two sums go to ax[r] and bd[r]. For NB = 4 and 8 lane l takes the
// blocks in the order J + l mod NB (the G stride is then 4 NB words: see bl_ldg, bl_rot).
template <typename T, int NB>
__device__ __forceinline__ void rows_t(const T *G, int ldg, const T *x, const T *du, int jx, int l,
                                       int g, int nx, T *ax, T *bd) {
  constexpr bool kRot = NB == 4 || NB == 8;
  for (int r = l; r < nx; r += g) {
    const T *row = G + r * ldg;
    V4<T> sa = zero4<T>(), sb = zero4<T>();
#pragma unroll
    for (int Js = 0; Js < NB; ++Js) {
      const int J = kRot ? ((Js + l) & (NB - 1)) : Js;
      const V4<T> gr = ld4(row + 4 * J), xv = ld4(x + 4 * J);
#pragma unroll
      for (int i = 0; i < 4; ++i) sa.v[i] += gr.v[i] * xv.v[i];
      if (J >= jx) {
        const V4<T> dv = ld4(du + 4 * J);
#pragma unroll
        for (int i = 0; i < 4; ++i) sb.v[i] += gr.v[i] * dv.v[i];
      }
    }
    ax[r] = (sa.v[0] + sa.v[1]) + (sa.v[2] + sa.v[3]);
    bd[r] = (sb.v[0] + sb.v[1]) + (sb.v[2] + sb.v[3]);
  }
}

template <typename T>
__device__ __forceinline__ void rows_rt(const T *G, int ldg, const T *x, const T *du, int jx,
                                        int l, int g, int nx, int nb, T *ax, T *bd) {
  for (int r = l; r < nx; r += g) {  // nb > 8: odd G stride, blocks in order
    const T *row = G + r * ldg;
    V4<T> sa = zero4<T>(), sb = zero4<T>();
    for (int J = 0; J < nb; ++J) {
      const V4<T> gr = ld4(row + 4 * J), xv = ld4(x + 4 * J);
#pragma unroll
      for (int i = 0; i < 4; ++i) sa.v[i] += gr.v[i] * xv.v[i];
      if (J >= jx) {
        const V4<T> dv = ld4(du + 4 * J);
#pragma unroll
        for (int i = 0; i < 4; ++i) sb.v[i] += gr.v[i] * dv.v[i];
      }
    }
    ax[r] = (sa.v[0] + sa.v[1]) + (sa.v[2] + sa.v[3]);
    bd[r] = (sb.v[0] + sb.v[1]) + (sb.v[2] + sb.v[3]);
  }
}

template <typename T>
__device__ __forceinline__ void rows(const T *G, int ldg, const T *x, const T *du, int jx, int l,
                                     int g, int nx, int nb, T *ax, T *bd) {
  switch (nb) {
    case 1: rows_t<T, 1>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 2: rows_t<T, 2>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 3: rows_t<T, 3>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 4: rows_t<T, 4>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 5: rows_t<T, 5>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 6: rows_t<T, 6>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 7: rows_t<T, 7>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    case 8: rows_t<T, 8>(G, ldg, x, du, jx, l, g, nx, ax, bd); break;
    default: rows_rt(G, ldg, x, du, jx, l, g, nx, nb, ax, bd); break;
  }
}

template <typename T>
__device__ inline T clampv(T x, T lo, T hi) {
  return x < lo ? lo : (x > hi ? hi : x);
}

// Momentum hat of four components of an iterate in global memory: cur + f (cur - prev).
template <typename T>
__device__ __forceinline__ V4<T> hat4(const T *cur, const T *prev, bool use_prev, T f) {
  V4<T> x = ldg4(cur);
  if (use_prev) {
    const V4<T> p = ldg4(prev);
#pragma unroll
    for (int i = 0; i < 4; ++i) x.v[i] += f * (x.v[i] - p.v[i]);
  }
  return x;
}

// kSets: compiled with the projection onto non-box input sets; the batches without them run the
// variant that has only the box.
template <typename T, bool kSets>
__global__ void __launch_bounds__(kThreads, 3) blk_kernel(Args<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int sDesc[4], sOk;
  __shared__ double sRed[kThreads / 32];
  T *sm = reinterpret_cast<T *>(smem_raw);
  constexpr int TS = (int)sizeof(T);
  const int tid = threadIdx.x;
  const unsigned nblocks = gridDim.x;
  Ctl *ctl = a.ctl;
  const int lti = a.L.lti;

  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par = 0u;
  bool pend = false;
  // Thread 0 fetches the next item (queue slot, list entry, item fields: three dependent global
  // reads) during the current item's last sub-chunk, one step per phase, so that it is known
  // when the item ends. nstate: 0 nothing fetched, 1 slot taken, 2 entry known, 3 ready (an item,
  // or -1 for a marked entry), 4 the queue is empty.
  int nstate = 0, nq = 0, nitem = 0, nj = 0, nka = 0, nkb = 0;

  int cl = 0;
  for (int it = 0; it < a.max_iters; ++it) {
    const int nact = *(volatile int *)&ctl->nlist[cl];
    bool ok = true;
    auto advance = [&]() {  // thread 0: one step of the next item's fetch
      if (nstate == 1) {
        if (nq < nact) { nitem = a.list[cl][nq]; nstate = 2; } else { nstate = 4; }
      } else if (nstate == 2) {
        if (nitem >= 0) { nj = a.item_inst[nitem]; nka = a.item_a[nitem]; nkb = a.item_b[nitem]; }
        nstate = 3;
      }
    };
    for (;;) {
      if (tid == 0) {
        if (nstate == 0) { nq = atomicAdd(&ctl->queue[it & 1], 1); nstate = 1; }
        while (nstate == 1 || nstate == 2) advance();
        sDesc[0] = nstate == 3 ? nitem : -2;  // -1: an entry of a stopped instance; -2: no more
        sDesc[1] = nj; sDesc[2] = nka; sDesc[3] = nkb;
        nstate = 0;
      }
      __syncthreads();
      const int item = sDesc[0], j = sDesc[1], ka = sDesc[2], kb = sDesc[3];
      __syncthreads();
      if (item == -2) break;
      if (item < 0) continue;
      // No stop check: the flags change only in the pass between iterations, which marks the
      // list entries of the instances it stops (-1) until a compaction removes them.
      const int nx = a.L.nx[j], nu = a.L.nu[j], N = a.L.N[j], n = nx + nu;
      const int g = bl_group(n), S = a.grp[j], P = S - 1;
      const int nP = bl_pad4(n), rec = bl_rec(n), nb = bl_nb(n);
      const int ldg = bl_ldg(n, TS), oE = bl_oE(nx, nu, TS), oH = bl_oH(nx, nu, TS);
      const int oM = bl_oM(nx, nu, TS), symW = bl_sym_words(n);
      const int W = a.L.W[j];
      const Regions R = regions(nx, nu, lti, TS, S);
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
      const int c0 = 4 * l;
      const bool own = c0 < n;
      // this group's scratch (only touched when grp < S): y / h / Abar xbar, w / B du, q, t, du
      T *scr = sm + R.scr + grp * 5 * nP;
      T *sY = scr, *sW = scr + nP, *sQ = scr + 2 * nP, *sT = scr + 3 * nP, *sDU = scr + 4 * nP;
      T *rB = sm;
      T *hB = sm + R.haloB;
      const T *ltiB = hB;  // stage-invariant: block 0 (H_k, k < N-1) then block 1 (H_{N-1})
      T *sQd = sm + R.prm, *sLo = sQd + nP, *sHi = sLo + nP;
      T cacc = (T)0;
      // Qbar diagonal and bounds of the instance into shared memory (first read after the
      // barrier that ends phase 1; the previous item's last read preceded its final barrier).
      for (int c = tid; c < nP; c += kThreads) {
        const bool in = c < n;
        sQd[c] = in ? qd[c] : (T)0;
        sLo[c] = in ? lo[c] : (T)0;
        sHi[c] = in ? hi[c] : (T)0;
      }

      // Copies of the sub-chunk that starts at stage k0 (thread 0 issues): the stage blocks
      // (stage-invariant instances: both blocks, once per item). A sub-chunk with nothing to
      // copy completes its phase with the arrival alone. (The shared-memory buffer the copies
      // overwrite was only read, and those reads precede the CTA barrier.)
      auto issue = [&](int k0, bool first) {
        const int cnt = min(P, kb - k0);
        const int la = (k0 + cnt < N) ? 1 : 0;  // the next stage: its G and e only
        const bool halo = first && ka > 0;
        const uint32_t blk_bytes = (uint32_t)((cnt * W + la * oH) * TS);
        uint32_t bytes = 0u;
        if (!lti) bytes += blk_bytes;
        if (halo && !lti) bytes += (uint32_t)(symW * TS);
        if (lti && first) bytes += (uint32_t)(2 * W * TS);
        mbar_expect_tx(&mbar, bytes);
        if (!lti) bulk_load(rB, blk + (int64_t)k0 * W, blk_bytes, &mbar);
        if (halo && !lti) bulk_load(hB, blk + (int64_t)(ka - 1) * W + oH, (uint32_t)(symW * TS), &mbar);
        if (lti && first) bulk_load(hB, blk, (uint32_t)(2 * W * TS), &mbar);
      };

      // L2 prefetch of the sub-chunk that starts at stage k0 (the same ranges as its copies):
      // its HBM reads overlap the current sub-chunk, and its copies then read L2.
      auto prefetch = [&](int k0) {
        const int cnt = min(P, kb - k0);
        const int la = (k0 + cnt < N) ? 1 : 0;
        const uint32_t it_bytes = (uint32_t)((cnt + la) * rec * TS);
        if (!lti) bulk_prefetch_l2(blk + (int64_t)k0 * W, (uint32_t)((cnt * W + la * oH) * TS));
        bulk_prefetch_l2(Ic + (int64_t)k0 * rec, it_bytes);
        if (use_prev) bulk_prefetch_l2(Ip + (int64_t)k0 * rec, it_bytes);
      };

      const int nsub = (kb - ka + P - 1) / P;
      if (tid == 0) issue(ka, true);
      pend = true;
      for (int sc = 0; sc < nsub; ++sc) {
        const int k0 = ka + sc * P;
        const int cnt = min(P, kb - k0);
        const bool la = k0 + cnt < N;
        if (sc > 0) {  // the single buffer is free after the previous sub-chunk's last barrier
          if (tid == 0) issue(k0, false);
          pend = true;
        }
        if (tid == 0 && sc + 1 < nsub) prefetch(k0 + P);
        // The reference of this group's stage (needed in phase 2) and the hats (phase 1 onwards)
        // do not come with the copies: their loads are issued before the wait.
        const int k = k0 + grp;
        V4<T> rf4 = zero4<T>();
        if (ref && grp < cnt && own) {
          const T *rk = ref + (int64_t)k * refstride;
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (c0 + i < n) rf4.v[i] = rk[c0 + i];
        }
        V4<T> zh = zero4<T>(), vh = zero4<T>(), th = zero4<T>(), bh = zero4<T>(), lh = zero4<T>();
        if ((grp < cnt || (grp == cnt && la)) && own) {
          const T *hc = Ic + (int64_t)k * rec + c0, *hp = Ip + (int64_t)k * rec + c0;
          zh = hat4(hc, hp, use_prev, f);
          vh = hat4(hc + nP, hp + nP, use_prev, f);
          lh = hat4(hc + 4 * nP, hp + 4 * nP, use_prev, f);
          if (grp < cnt) {
            th = hat4(hc + 2 * nP, hp + 2 * nP, use_prev, f);
            bh = hat4(hc + 3 * nP, hp + 3 * nP, use_prev, f);
          }
        }
        // Every thread waits on the copies itself (bounded), so no CTA barrier is needed here;
        // a timeout seen by any thread ends the item for the whole CTA at the barrier after
        // phase 1.
        const bool arrived = mbar_wait(&mbar, par, ctl);
        if (arrived) {
          par ^= 1u;
          pend = false;
        } else {
          ok = false;  // the copy may still be in flight: it stays pending for the exit wait
        }
        if (tid == 0 && sc == nsub - 1 && nstate == 0) {
          nq = atomicAdd(&ctl->queue[it & 1], 1);  // the next item's slot; used after the barrier
          nstate = 1;
        }
        T *Xc = sm + R.X + (sc & 1) * S * nP;
        T *Xn = sm + R.X + ((sc & 1) ^ 1) * S * nP;
        const bool stage = arrived && grp < cnt;           // stage k of this sub-chunk
        const bool look = arrived && grp == cnt && la;     // the next stage: q only
        const bool hgrp = arrived && sc == 0 && ka > 0 && grp == S - 1;  // recomputes xbar_a
        const T *Gk = lti ? ltiB : rB + grp * W;

        // ---- phase 1: y and w from the hats; q and t in one pass over G_k; du = M t ----
        V4<T> e4 = zero4<T>(), y4 = zero4<T>(), w4 = zero4<T>();
        if ((stage || look) && own) {
          if (c0 < nx) e4 = ld4(Gk + oE + c0);  // zero beyond nx (padding)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            y4.v[i] = zh.v[i] - vh.v[i] + lh.v[i] - e4.v[i];
            w4.v[i] = vh.v[i] - bh.v[i];
          }
          st4(sY + c0, y4);
          st4(sW + c0, w4);
          st4(sDU + c0, zero4<T>());
        }
        if (sc == 0 && ka == 0)
          for (int c = tid; c < nP; c += kThreads) Xc[c] = c < n ? a.xb0[a.L.off_n[j] + c] : (T)0;
        __syncwarp();
        if ((stage || look) && own) {
          V4<T> qv = zero4<T>(), tv = zero4<T>();
          const T *gc = Gk + c0;
          int r = 0;
          for (; r + 3 < nx; r += 4) {
            const V4<T> yv = ld4(sY + r), wv = ld4(sW + r);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const V4<T> gr = ld4(gc + (r + u) * ldg);
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                qv.v[i] += gr.v[i] * yv.v[u];
                tv.v[i] += gr.v[i] * wv.v[u];
              }
            }
          }
          for (; r < nx; ++r) {
            const T yr = sY[r], wr = sW[r];
            const V4<T> gr = ld4(gc + r * ldg);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              qv.v[i] += gr.v[i] * yr;
              tv.v[i] += gr.v[i] * wr;
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (c0 + i >= nx) {  // the identity rows of Abar, and w_u in t
              qv.v[i] += y4.v[i];
              tv.v[i] += w4.v[i];
            }
          st4(sQ + c0, qv);
          st4(sT + c0, tv);
        }
        __syncwarp();
        if (stage)
          for (int jj = l; jj < nu; jj += g) sDU[nx + jj] = sym_wrapped(Gk + oM, sT + nx, nu, jj);
        if (!__syncthreads_and(arrived)) { ok = false; break; }  // uniform across the CTA
        if (tid == 0) advance();

        // ---- phase 2: h_k (with q_{k+1} of the next group) and xbar_{k+1} = H_k h_k ----
        if (stage && own) {
          V4<T> qn = zero4<T>();
          if (k + 1 < N) qn = ld4(scr + 5 * nP + 2 * nP + c0);  // the next group's q
          const V4<T> qd4 = ld4(sQd + c0);
          // h is zero beyond n, where qd, the hats, q and the reference are zero
          V4<T> h;
#pragma unroll
          for (int i = 0; i < 4; ++i) h.v[i] = qd4.v[i] * rf4.v[i] + rho * (zh.v[i] - th.v[i] + qn.v[i]);
          st4(sY + c0, h);
        }
        if (hgrp && own) {  // h_{a-1} from the halo hats and q_a (group 0)
          const T *hm = Ic + (int64_t)(ka - 1) * rec + c0, *pm = Ip + (int64_t)(ka - 1) * rec + c0;
          const V4<T> zm = hat4(hm, pm, use_prev, f);
          const V4<T> tm = hat4(hm + 2 * nP, pm + 2 * nP, use_prev, f);
          const V4<T> qa = ld4(sm + R.scr + 2 * nP + c0);
          const V4<T> qd4 = ld4(sQd + c0);
          V4<T> h;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = c0 + i;
            const T rf = (ref && c < n) ? ref[(int64_t)(ka - 1) * refstride + c] : (T)0;
            h.v[i] = qd4.v[i] * rf + rho * (zm.v[i] - tm.v[i] + qa.v[i]);
          }
          st4(sY + c0, h);
        }
        __syncwarp();
        if ((stage || hgrp) && l < nb) {
          const T *Hb = stage ? (lti ? ltiB + ((k < N - 1) ? 0 : W) + oH : rB + grp * W + oH)
                              : (lti ? ltiB + oH : hB);
          const V4<T> x = sym_blocks(Hb, sY, nb, l);
          if (stage) {
            st4(Xc + (grp + 1) * nP + c0, x);
            if (grp + 1 == cnt) st4(Xn + c0, x);  // row 0 of the next sub-chunk
          } else {
            st4(Xc + c0, x);
          }
        }
        __syncthreads();
        if (tid == 0) advance();

        // ---- phase 3: Abar xbar_k and B du by rows; steps 2-4 on the owned components ----
        if (stage)  // jx = nx / 4: the first column block that holds input columns
          rows(Gk, ldg, Xc + grp * nP, sDU, nx >> 2, l, g, nx, nb, sY, sW);
        __syncwarp();
        {
          // w of the owned components (stage && own), the input part projected onto a non-box
          // set U (warp-wide; the kind is the same for the CTA's item), then steps 2-4.
          const bool mine = stage && own;
          T wv[4] = {(T)0, (T)0, (T)0, (T)0}, gv[4], axv[4], bdv[4], eev[4], xnv[4];
          T av[4] = {(T)0, (T)0, (T)0, (T)0};
          int cv[4] = {-1, -1, -1, -1};
          if (mine) {
            const T *xk = Xc + grp * nP, *xk1 = Xc + (grp + 1) * nP;
            const V4<T> x1 = ld4(xk1 + c0), x0 = ld4(xk + c0), du4 = ld4(sDU + c0);
            const V4<T> ax4 = ld4(sY + c0), bd4 = ld4(sW + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int c = c0 + i;
              if (c < n) {
                const bool xs = c < nx;
                axv[i] = xs ? ax4.v[i] : x0.v[i];
                bdv[i] = xs ? bd4.v[i] : du4.v[i];
                eev[i] = e4.v[i];
                xnv[i] = x1.v[i];
                gv[i] = bdv[i] + bh.v[i] - axv[i] - eev[i] + lh.v[i];
                wv[i] = ((T)2 * (xnv[i] + th.v[i] + axv[i] + eev[i] - lh.v[i]) + gv[i]) / (T)3;
                cv[i] = c;
                if (ukind == uset::kUsetHalfspace && !xs) av[i] = ua[c];
              }
            }
          }
          if (kSets && ukind != uset::kUsetBox)
            uset::project_inputs<T, 4>(ukind, ur, av, wv, cv, nx, n, g,
                                       [](int jj) { return jj >> 2; }, [](int jj) { return jj & 3; });
          if (mine) {
          const V4<T> lo4 = ld4(sLo + c0), hi4 = ld4(sHi + c0);
          V4<T> oz, ov, ot, ob, ol;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = c0 + i;
            if (c < n) {
              const T ax = axv[i], bd = bdv[i], ee = eev[i], xn = xnv[i], gam = gv[i];
              const T z = (c < nx || ukind == uset::kUsetBox) ? clampv(wv[i], lo4.v[i], hi4.v[i])
                                                              : wv[i];
              const T v = (T)0.5 * (z + gam);
              const T tt = th.v[i] + xn - z;
              const T be = bh.v[i] + bd - v;
              const T lam = lh.v[i] + z - ax - v - ee;
              const T d1 = tt - th.v[i], d2 = be - bh.v[i], d3 = lam - lh.v[i];
              const T d4 = z - zh.v[i], d5 = v - vh.v[i], d6 = d4 - d5;
              cacc += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
              oz.v[i] = z; ov.v[i] = v; ot.v[i] = tt; ob.v[i] = be; ol.v[i] = lam;
            } else {
              oz.v[i] = ov.v[i] = ot.v[i] = ob.v[i] = ol.v[i] = (T)0;
            }
          }
          T *o = In + (int64_t)k * rec + c0;
          st4(o, oz);
          st4(o + nP, ov);
          st4(o + 2 * nP, ot);
          st4(o + 3 * nP, ob);
          st4(o + 4 * nP, ol);
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
        for (int w = 0; w < kThreads / 32; ++w) part += sRed[w];
        a.cpart[item] = part;  // steps 5-7 run in the pass after the barrier
      }
    }
    if (blockIdx.x == 0 && tid == 0) ctl->queue[(it + 1) & 1] = 0;
    if (!ls::grid_sync(ctl, nblocks, &sOk)) break;
    if (!ls::finish_pass(a, it, cl, nblocks, &sOk)) break;
    if (*(volatile int *)&ctl->active <= 0) break;
    if (!ls::compact(a, cl, nact, &sOk, reinterpret_cast<int *>(sRed))) break;
  }
  // Never leave a bulk copy in flight into shared memory: wait (bounded) for the pending phase.
  if (pend) {
    long long k = 0;
    while (!mbar_try_wait(&mbar, par) && ++k < kWaitLimit) {
    }
  }
}

}  // namespace

int blk_threads() { return kThreads; }

int64_t blk_region_words(int nx, int nu, int lti, int precision, int S) {
  return regions(nx, nu, lti, precision == 0 ? 4 : 8, S).total;
}

cudaError_t blk_configure(int precision, size_t smem, int *blocks_per_sm) {
  cudaError_t rc;
  if (precision == 0) {
    rc = cudaFuncSetAttribute(blk_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, blk_kernel<float, false>, kThreads, smem);
  } else {
    rc = cudaFuncSetAttribute(blk_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, blk_kernel<double, false>, kThreads, smem);
  }
  return rc;
}

cudaError_t launch_blk(const AdmmLaunch &s, int precision, size_t smem, cudaStream_t stream) {
  if (precision == 0) {
    ls::Args<float> a = ls::make_args<float>(s);
    void *params[] = {&a};
    const void *k = s.uset_kind ? (const void *)blk_kernel<float, true> : (const void *)blk_kernel<float, false>;
    return ls::launch_sequence<float>(s, a, k, params, smem, stream);
  }
  ls::Args<double> a = ls::make_args<double>(s);
  void *params[] = {&a};
  const void *k = s.uset_kind ? (const void *)blk_kernel<double, true> : (const void *)blk_kernel<double, false>;
  return ls::launch_sequence<double>(s, a, k, params, smem, stream);
}

}  // namespace pimpc

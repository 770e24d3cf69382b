// lockstep.cuh -- the persistent, lock-step frame shared by the solve kernels (internal).
//
// One cooperative launch runs every iteration of every instance. In iteration i each CTA pulls
// work items (instance j, stage range) from a queue and runs the iteration on them; a bounded
// grid barrier separates iterations. Each item stores its share of c^{i+1}; after the barrier a
// pass over the instances still iterating (one thread each) sums the shares and applies
// Algorithm 1 steps 5-7 (stop test, momentum or restart), and a second barrier publishes the
// decisions; stopped instances then leave the queue by stream compaction.
#pragma once
#include <math.h>

#include "launch.h"

namespace pimpc {
namespace ls {

constexpr long long kWaitLimit = 1ll << 22;  // bounded polls of the grid barrier / mbarriers

template <typename T>
struct Args {
  Layout L;
  const T *blk;
  T *it[3];
  const T *qd, *ref;
  int ref_per_stage;
  const T *lo, *hi, *xb0;
  double rho, eps, eta;
  int max_iters, accel;
  const unsigned char *mask;
  int mask_len;
  const int *item_inst, *item_a, *item_b;
  int nitems;
  const int *nitems_inst;   // [batch] coarse counts, then [batch] fine counts
  const int *item_first;    // [batch] first coarse item, then [batch] first fine item (null:
                            // the items accumulate c through finish_item instead)
  double *cpart;            // [items] each item's share of c^{i+1} in the current iteration
  const int *list_init;     // [coarse items] the starting order of the active list (null:
                            // item order), longest first
  int *ccount;              // [grid] per-CTA counts of the order-keeping compaction (null: the
                            // compaction keeps no order)
  int *pos_of;              // [items] position of each item in the active list: the entries of
                            // a stopped instance are marked -1 there, and the list is compacted
                            // once they are a 32nd of it (null: compacted every iteration)
  int nfine_base, nfine;    // fine items: nfine of them from nfine_base (0: none)
  int fine_switch;          // switch to them below fine_switch x grid active coarse items
  int *list[2];
  Ctl *ctl;
  int *base;
  InstState *st;
  double *alpha, *cprev, *coef, *cacc;
  int *ndone, *stop;
  int capI;
  const double *coef_tab;  // momentum factor of the m-th consecutive momentum step (resident)
  const int *grp;          // blocked kernel: lane groups per sub-chunk of each instance
  const int *ferr;         // [batch] factorisation failure flags (may be null)
  int stall_win;           // > 0: stop an instance whose c has stalled (see stalled())
  const int *uset_kind;    // input set of each instance (null: all boxes), radius, normal
  const T *uset_r, *uset_a;
  double stall_fac, stall_below, stall_rel;
  double *cbest;
  int *itbest, *itfirst;
};

// Iterate element (vector b in {z, v, theta, beta, lambda}, component c) of stage k (its own
// copy). Plain layout: stage-major with stride n5p. Tiled layout: tiles of 32 stages,
// element-major inside a tile (one 128-byte line per element for 32 stages in FP32). Halo
// tiles: tw slots per tile (see pimpc_internal.cuh). Blocked layout: stage-major, every vector
// padded to a multiple of 4 (n5p is not used). Layout 4 (tensor-core schedule): tiles of 128
// stages; inside a tile, for every vector and every group of 4 components of the padded vector
// (x part and u part each rounded up to 16), the 128 stages' 4 components contiguous (one
// 16-byte load per stage); tw passes nx for it (layout_aux).
__host__ __device__ inline int64_t iter_index(int tiled, int tw, int n, int n5p, int k, int b,
                                              int c) {
  if (tiled == 1) return (int64_t)(k >> 5) * (32 * 5 * n) + (int64_t)(b * n + c) * 32 + (k & 31);
  if (tiled == 2) {
    int t, s;
    halo_slot(tw, k, t, s);
    return (int64_t)t * tile_iter_words(tw, n) + (int64_t)(b * n + c) * tw + s;
  }
  if (tiled == 3) return (int64_t)k * bl_rec(n) + b * bl_pad4(n) + c;
  if (tiled == 4) {  // tw carries nx here: vectors padded to (nx, nu) rounded up to 16 each
    const int nx = tw, nxp = (nx + 15) & ~15, np = nxp + ((n - nx + 15) & ~15);
    const int p = c < nx ? c : nxp + (c - nx);
    return (int64_t)(k >> 7) * (128 * 5 * np) + (int64_t)(b * np + (p & ~3)) * 128 + (k & 127) * 4 +
           (p & 3);
  }
  return (int64_t)k * n5p + b * n + c;
}

// The per-instance parameter iter_index takes besides n: the halo tile width (layout 2) or nx
// (layout 4).
__host__ __device__ inline int layout_aux(const Layout &L, int j) {
  return L.tiled == 2 ? L.tw[j] : (L.tiled == 4 ? L.nx[j] : 0);
}

__host__ __device__ inline int iter_stride_plain(int n, int tsize) {
  const int q = 16 / tsize;
  return (5 * n + q - 1) / q * q;
}

// Bounded grid barrier; all CTAs of the cooperative launch are co-resident.
__device__ inline bool grid_sync(Ctl *c, unsigned nblocks, int *sOk) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = &c->bar_gen;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      c->bar_count = 0;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const int lim = *(volatile int *)&c->bar_limit;
      const long long limit = lim > 0 ? (long long)lim : kWaitLimit;
      long long k = 0;
      while (*gen == g) {
        if (++k > limit || *(volatile int *)&c->err) { ok = 0; break; }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (!ok) atomicExch(&c->err, 1);
    *sOk = ok && (*(volatile int *)&c->err == 0);
  }
  __syncthreads();
  return *sOk != 0;
}

// Per-instance state that steps 5-7 read. It does not depend on c^{i+1}, so the pass over the
// instances loads it in the same round as the item counts, before the shares of c arrive.
struct StepState {
  double cprev, alpha, cbest;
  int momentum, itfirst, itbest;
};

template <typename T>
__device__ inline StepState load_step_state(const Args<T> &a, int j) {
  StepState q;
  q.cprev = a.cprev[j];
  q.alpha = a.alpha[j];
  q.momentum = a.st[j].momentum;
  if (a.stall_win > 0) {
    q.cbest = a.cbest[j];
    q.itfirst = a.itfirst[j];
    q.itbest = a.itbest[j];
  } else {
    q.cbest = 0.0;
    q.itfirst = q.itbest = 0;
  }
  return q;
}

// The floor of the iteration's arithmetic: since c^{i+1} first came below stall_below (at
// iteration i0), it has not fallen below stall_fac times the best c for max(stall_win,
// stall_rel i0) iterations. In FP32 c stops decreasing once the rounding of the iterates
// dominates their change; plateaus of the accelerated iteration far above that floor do not
// count, and the window grows with i0 because an instance that converges slowly (large i0)
// keeps improving its iterates for longer after its c has levelled off. Updates the best c.
// Called by one thread, only for c <= stall_below; q holds the instance's state as loaded.
template <typename T>
__device__ inline bool stalled(const Args<T> &a, int j, int it, double c, StepState &q) {
  if (q.itfirst < 0) {
    q.itfirst = it;
    a.itfirst[j] = it;
  }
  if (c < a.stall_fac * q.cbest) {
    q.cbest = c;
    q.itbest = it;
    a.cbest[j] = c;
    a.itbest[j] = it;
    return false;
  }
  const double win = fmax((double)a.stall_win, a.stall_rel * (double)q.itfirst);
  return (double)(it - q.itbest) >= win;
}

// Steps 5-7 of instance j given the sum s of its squared step-4 terms (c^{i+1} = rho s): the stop
// tests, then the momentum decision and factor. Called by one thread; q is the instance's state
// (load_step_state), written back where it changes.
template <typename T>
__device__ inline bool apply_steps(const Args<T> &a, int j, int it, double s, StepState q) {
  const double c = a.rho * s;
  InstState &st = a.st[j];
  st.iters = it + 1;
  st.c = c;
  int stop = 0;
  if (!isfinite(c)) {
    st.status = kNonFinite; stop = 1;
  } else if (c <= a.eps) {
    st.status = kConverged; stop = 1;
  } else if (a.stall_win > 0 && c <= a.stall_below && stalled(a, j, it, c, q)) {
    st.status = kStalled; stop = 1;
  } else if (it + 1 >= a.max_iters) {
    st.status = kMaxIter; stop = 1;
  } else {
    int take = 0;
    if (a.accel) {
      if (a.mask && it < a.mask_len) take = a.mask[(int64_t)j * a.mask_len + it] != 0;
      else take = c <= a.eta * q.cprev;
    }
    if (take) {
      const double al = q.alpha;
      const double an = 0.5 + 0.5 * sqrt(1.0 + 4.0 * al * al);
      a.coef[j] = (al - 1.0) / an;
      a.alpha[j] = an;
      if (al != 1.0) st.momentum = q.momentum + 1;
    } else {
      a.alpha[j] = 1.0;
      a.coef[j] = 0.0;
    }
    a.cprev[j] = c;
  }
  if (stop) {
    a.stop[j] = 1;
    a.base[j] = (a.base[j] + it + 1) % 3;  // the buffer holding the final iterate
    atomicSub(&a.ctl->active, 1);
    atomicExch(&a.ctl->stopped, 1);
  }
  return stop != 0;
}

// Step 4's reduction is finished by the caller; this adds the item's share of c^{i+1} and, for
// the instance's last item of the iteration, applies steps 5-7. Called by one thread.
template <typename T>
__device__ inline void finish_item(const Args<T> &a, int j, int it, double part) {
  atomicAdd(&a.cacc[j], part);
  __threadfence();
  const int done = atomicAdd(&a.ndone[j], 1);
  const int fine = *(volatile int *)&a.ctl->fine;
  if (done != a.nitems_inst[j + (fine ? a.L.batch : 0)] - 1) return;
  __threadfence();
  const double s = __longlong_as_double((long long)atomicExch((unsigned long long *)&a.cacc[j], 0ull));
  a.ndone[j] = 0;
  apply_steps(a, j, it, s, load_step_state(a, j));
}

// After the iteration's grid barrier: steps 5-7 for every instance still iterating, from the
// shares of c^{i+1} its items stored in cpart (summed in item order, so c does not depend on
// which CTA finished last), then a grid barrier so that every CTA sees the decisions (stop,
// momentum factor) before the next iteration. The items themselves only store their share:
// no atomics or fences on the item path. Every item of an instance still iterating runs in
// every iteration (the active list holds all of them), so the shares are complete.
// An instance that stops has its entries in the active list (cl) marked -1 when pos_of is kept.
// The loads that do not depend on each other (the stop flag, both item ranges, the state of
// steps 5-7) are issued together, so that the pass waits on two rounds of loads: those and the
// shares of c.
template <typename T>
__device__ inline bool finish_pass(const Args<T> &a, int it, int cl, unsigned nblocks, int *sOk) {
  const int fine = *(volatile int *)&a.ctl->fine;
  const int stride = (int)nblocks * blockDim.x;
  const int B = a.L.batch;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B; j += stride) {
    const int stopped = *(volatile int *)&a.stop[j];
    const int f0 = a.item_first[j], n0 = a.nitems_inst[j];
    const int f1 = a.item_first[j + B], n1 = a.nitems_inst[j + B];
    const StepState q = load_step_state(a, j);
    if (stopped) continue;
    const int first = fine ? f1 : f0, cnt = fine ? n1 : n0;
    double s = 0.0;
    for (int i = 0; i < cnt; ++i) s += __ldcg(a.cpart + first + i);
    if (apply_steps(a, j, it, s, q) && a.pos_of) {
      for (int i = 0; i < cnt; ++i) a.list[cl][__ldcg(a.pos_of + first + i)] = -1;
      atomicAdd(&a.ctl->stale, cnt);
    }
  }
  return grid_sync(a.ctl, nblocks, sOk);
}

// Sum over the CTA (every thread gets the total); red holds blockDim.x / 32 ints of scratch.
__device__ inline int block_sum(int v, int *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// After the iteration barrier: drop the items of stopped instances from the active list. When
// the active coarse items no longer cover the grid several times over (few instances left,
// each item run by one CTA one sub-chunk after the other, the last items of an iteration
// leaving most CTAs idle), the list is rebuilt from the fine items of the active instances
// instead, so that their sub-chunks spread over the CTAs. Returns false if a barrier
// failed. Uniform control flow across the grid (every CTA reads the same nact, stopped, fine).
// red: shared scratch of at least blockDim.x / 32 ints (the kernel's reduction buffer, free
// between iterations).
template <typename T>
__device__ inline bool compact(const Args<T> &a, int &cl, int nact, int *sOk, int *red) {
  Ctl *ctl = a.ctl;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const unsigned nblocks = gridDim.x;
  const bool go_fine =
      a.nfine > 0 && !*(volatile int *)&ctl->fine && nact < a.fine_switch * (int)nblocks;
  const int stopped = *(volatile int *)&ctl->stopped;
  if (!stopped && !go_fine) return true;
  if (a.pos_of && !go_fine) {  // marked entries are skipped: compact once they are a 32nd
    const int stale = *(volatile int *)&ctl->stale;
    if (stale > 0 && stale * 32 < nact) return true;
  }
  const int src = cl, dst = cl ^ 1;
  const int total = go_fine ? a.nfine : nact;
  auto entry = [&](int qi, int &item) {  // the qi-th source entry and whether it stays
    item = go_fine ? a.nfine_base + qi : a.list[src][qi];
    return item >= 0 && *(volatile int *)&a.stop[a.item_inst[item]] == 0;
  };
  if (a.ccount) {
    // Order-keeping: CTA b takes a contiguous range of the source list, counts what stays,
    // and after a barrier writes it at the sum of the counts of the CTAs before it, so the list
    // keeps its longest-first order (the queue then hands out the long items first).
    const int per = (total + (int)nblocks - 1) / (int)nblocks;
    const int q0 = min(total, (int)blockIdx.x * per), q1 = min(total, q0 + per);
    int kept = 0, item;
    for (int qi = q0 + tid; qi < q1; qi += nthreads) kept += entry(qi, item) ? 1 : 0;
    kept = block_sum(kept, red);
    if (tid == 0) a.ccount[blockIdx.x] = kept;
    if (!grid_sync(ctl, nblocks, sOk)) return false;
    int before = 0, all = 0;
    for (int b = tid; b < (int)nblocks; b += nthreads) {
      const int c = __ldcg(a.ccount + b);
      all += c;
      if (b < (int)blockIdx.x) before += c;
    }
    before = block_sum(before, red);
    all = block_sum(all, red);
    for (int c0 = q0; c0 < q1; c0 += nthreads) {
      const int qi = c0 + tid;
      const int keep = qi < q1 && entry(qi, item);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      __syncthreads();
      if ((tid & 31) == 0) red[tid >> 5] = __popc(m);
      __syncthreads();
      int wbase = 0;
      for (int w = 0; w < (tid >> 5); ++w) wbase += red[w];
      if (keep) {
        const int pos = before + wbase + __popc(m & ((1u << (tid & 31)) - 1u));
        a.list[dst][pos] = item;
        if (a.pos_of) a.pos_of[item] = pos;
      }
      int chunk = 0;
      for (int w = 0; w < (nthreads >> 5); ++w) chunk += red[w];
      before += chunk;
    }
    // Everyone read nlist[src], stopped and fine before the barrier above; the barrier below
    // publishes the new list with its length and the reset flags.
    if (blockIdx.x == 0 && tid == 0) {
      ctl->nlist[dst] = all;
      ctl->nlist[src] = 0;
      ctl->stopped = 0;
      ctl->stale = 0;
      if (go_fine) ctl->fine = 1;
    }
    cl = dst;
    return grid_sync(ctl, nblocks, sOk);
  } else {
    for (int b0 = blockIdx.x * nthreads; b0 < total; b0 += nblocks * nthreads) {
      const int qi = b0 + tid;
      int keep = 0, item = 0;
      if (qi < total) keep = entry(qi, item);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      int wbase = 0;
      if ((tid & 31) == 0 && m) wbase = atomicAdd(&ctl->nlist[dst], __popc(m));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (keep) a.list[dst][wbase + __popc(m & ((1u << (tid & 31)) - 1u))] = item;
    }
  }
  if (!grid_sync(ctl, nblocks, sOk)) return false;
  cl = dst;
  if (blockIdx.x == 0 && tid == 0) {
    ctl->nlist[src] = 0;
    ctl->stopped = 0;
    if (go_fine) ctl->fine = 1;
  }
  return grid_sync(ctl, nblocks, sOk);
}

// One thread per instance (and per item): reset the per-instance state before a solve.
template <typename T>
__global__ void solve_init_kernel(Args<T> a, int warm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.L.batch) {
    if (warm == 2) a.base[j] = (a.base[j] + 1) % 3;  // the shifted copy is written there
    a.alpha[j] = 1.0;
    a.cprev[j] = 1.0;
    a.coef[j] = 0.0;
    a.cacc[j] = 0.0;
    a.ndone[j] = 0;
    a.stop[j] = a.max_iters <= 0 ? 1 : 0;
    if (a.stall_win > 0) {
      a.cbest[j] = INFINITY;
      a.itbest[j] = 0;
      a.itfirst[j] = -1;
    }
    InstState s;
    s.iters = 0; s.status = kMaxIter; s.momentum = 0; s.pad = 0; s.c = 0.0;
    a.st[j] = s;
  }
  if (j < a.nitems) {
    const int item = a.list_init ? a.list_init[j] : j;
    a.list[0][j] = item;
    if (a.pos_of) a.pos_of[item] = j;
  }
}

// Starting iterates: zero (cold start) or the previous solve's iterates shifted one stage.
template <typename T>
__global__ void prepare_kernel(Args<T> a, int warm, const int *old_base) {
  const int j = blockIdx.y;
  const int n = a.L.nx[j] + a.L.nu[j], N = a.L.N[j];
  const int tiled = a.L.tiled;
  const int tw = layout_aux(a.L, j);
  const int n5p = iter_stride_plain(n, (int)sizeof(T));
  const int64_t ib = a.L.Ni[j];
  T *dst = a.it[a.base[j]] + ib;
  const T *src = a.it[old_base[j]] + ib;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * 5 * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / (5 * n)), r = (int)(t - (int64_t)k * 5 * n);
    const int b = r / n, c = r - b * n;
    T v = (T)0;
    if (warm != 0) {
      const int ks = k + 1 < N ? k + 1 : N - 1;
      v = src[iter_index(tiled, tw, n, n5p, ks, b, c)];
    }
    dst[iter_index(tiled, tw, n, n5p, k, b, c)] = v;
    if (tiled == 2) {  // the copies in the neighbouring tiles' halo slots
      int tt[2], ss[2];
      const int m = halo_copies(tw, N, k, tt, ss);
      for (int q = 0; q < m; ++q)
        dst[(int64_t)tt[q] * tile_iter_words(tw, n) + (int64_t)(b * n + c) * tw + ss[q]] = v;
    }
  }
}

// u_k and x_{k+1} from z_{k+1} of the final iterate; instances whose stage cache met a
// non-positive pivot are reported as PIMPC_FACTOR_FAILED, instances the launch did not finish
// (a timed-out wait) as PIMPC_TIMEOUT.
template <typename T>
__global__ void output_kernel(Args<T> a, double *u_out, double *x_out) {
  const int j = blockIdx.y;
  const int nx = a.L.nx[j], nu = a.L.nu[j], n = nx + nu, N = a.L.N[j];
  const int n5p = iter_stride_plain(n, (int)sizeof(T));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (a.ferr && a.ferr[j]) a.st[j].status = kFactorFailed;
    else if (!a.stop[j]) a.st[j].status = kTimeout;
  }
  const T *z = a.it[a.base[j]] + a.L.Ni[j];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / n), c = (int)(t - (int64_t)k * n);
    const int tw = layout_aux(a.L, j);
    const double v = (double)z[iter_index(a.L.tiled, tw, n, n5p, k, 0, c)];
    if (c < nx) {
      if (x_out) x_out[a.L.Nnx[j] + (int64_t)k * nx + c] = v;
    } else if (u_out) {
      u_out[a.L.Nnu[j] + (int64_t)k * nu + (c - nx)] = v;
    }
  }
}

template <typename T>
Args<T> make_args(const AdmmLaunch &s) {
  Args<T> a;
  a.L = s.L;
  a.blk = (const T *)s.blk;
  for (int b = 0; b < 3; ++b) a.it[b] = (T *)s.it[b];
  a.qd = (const T *)s.qd;
  a.ref = (const T *)s.ref;
  a.ref_per_stage = s.ref_per_stage;
  a.lo = (const T *)s.lo;
  a.hi = (const T *)s.hi;
  a.xb0 = (const T *)s.xb0;
  a.rho = s.rho; a.eps = s.eps; a.eta = s.eta;
  a.max_iters = s.max_iters; a.accel = s.accel;
  a.mask = s.mask; a.mask_len = s.mask_len;
  a.item_inst = s.item_inst; a.item_a = s.item_a; a.item_b = s.item_b;
  a.nitems = s.nitems; a.nitems_inst = s.nitems_inst;
  a.item_first = s.item_first; a.cpart = s.cpart;
  a.list_init = s.list_init; a.ccount = s.ccount; a.pos_of = s.pos_of;
  a.nfine_base = s.nfine_base; a.nfine = s.nfine; a.fine_switch = s.fine_switch;
  a.list[0] = s.list0; a.list[1] = s.list1;
  a.ctl = s.ctl;
  a.base = s.base; a.st = s.st;
  a.alpha = s.alpha; a.cprev = s.cprev; a.coef = s.coef; a.cacc = s.cacc;
  a.ndone = s.ndone; a.stop = s.stop;
  a.capI = 0;
  a.coef_tab = s.coef_tab;
  a.grp = s.grp;
  a.ferr = s.ferr;
  a.stall_win = s.stall_win;
  a.uset_kind = s.uset_kind;
  a.uset_r = (const T *)s.uset_r;
  a.uset_a = (const T *)s.uset_a;
  a.stall_fac = s.stall_fac;
  a.stall_below = s.stall_below;
  a.stall_rel = s.stall_rel;
  a.itfirst = s.itfirst;
  a.cbest = s.cbest;
  a.itbest = s.itbest;
  return a;
}

// The launch sequence of one solve: per-instance reset, starting iterates, the persistent
// kernel (cooperative), outputs.
template <typename T>
cudaError_t launch_sequence(const AdmmLaunch &s, Args<T> &a, const void *kernel, void **params,
                            size_t smem, cudaStream_t stream) {
  cudaError_t rc = cudaMemsetAsync(s.ctl, 0, sizeof(Ctl), stream);
  if (rc != cudaSuccess) return rc;
  rc = cudaMemcpyAsync(s.old_base, s.base, sizeof(int) * s.L.batch, cudaMemcpyDeviceToDevice, stream);
  if (rc != cudaSuccess) return rc;
  const int n_init = s.L.batch > s.nitems ? s.L.batch : s.nitems;
  solve_init_kernel<T><<<(n_init + 255) / 256, 256, 0, stream>>>(a, s.warm);
  if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
  if (s.warm != 1) {
    prepare_kernel<T><<<dim3(8, s.L.batch), 256, 0, stream>>>(a, s.warm, s.old_base);
    if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
  }
  set_control_kernel<<<1, 1, 0, stream>>>(s.ctl, s.nitems, s.L.batch, s.bar_limit);
  if ((rc = cudaGetLastError()) != cudaSuccess) return rc;
  if (s.max_iters > 0) {
    rc = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) return rc;
    // Cooperative launch (all CTAs co-resident: the grid barrier relies on it), issued through
    // cudaLaunchKernelExC so that it can also be recorded into a CUDA graph.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s.grid);
    cfg.blockDim = dim3(s.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    rc = cudaLaunchKernelExC(&cfg, kernel, params);
    if (rc != cudaSuccess) return rc;
  }
  output_kernel<T><<<dim3(4, s.L.batch), 256, 0, stream>>>(a, s.u_out, s.x_out);
  return cudaGetLastError();
}

}  // namespace ls
}  // namespace pimpc

// api.cu -- the C ABI declared in include/pimpc.h: solver object, validation, host/device
// marshalling and the launch sequence of each call. Every piece of arithmetic runs in the
// kernels of factorise.cu, admm.cu, models.cu, adjoint.cu and misc.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "launch.h"
#include "pimpc.h"
#include "solver.h"

using namespace pimpc;

namespace pimpc {
cudaError_t launch_unpack_state(const InstState *st, int batch, int *iters, double *c,
                                int *status, int *momentum, cudaStream_t stream);
cudaError_t launch_copy_iterates(const Layout &Ls, void *const *its, const int *base_s, int prec_s,
                                 const Layout &Ld, void *const *itd, const int *base_d,
                                 cudaStream_t stream);
cudaError_t launch_add_state(InstState *st, const InstState *polish, int batch, cudaStream_t stream);
cudaError_t launch_fill(double *dst, int64_t count, double value, cudaStream_t stream);
}  // namespace pimpc

namespace {
thread_local std::string g_create_error;
}

namespace pimpc {

void set_thread_error(const std::string &msg) { g_create_error = msg; }

int fail(pimpc_solver *s, int code, const std::string &msg) {
  if (s) s->err = msg;
  return code;
}

// The resident kernel's table of momentum factors, long enough for max_iters iterations
// (computed on the device once per growth; not inside a stream capture).
int ensure_coef_table(pimpc_solver *s) {
  if (s->sched.family != 3 || s->coef_len >= s->max_iters + 1) return PIMPC_OK;
  const int len = std::max(s->max_iters + 1, 1024);
  if (s->coef_tab) cudaFree(s->coef_tab);
  s->coef_tab = nullptr;
  s->coef_len = 0;
  PIMPC_CHECK(s, cudaMalloc(&s->coef_tab, sizeof(double) * len), "momentum table");
  PIMPC_CHECK(s, launch_coef_table(s->coef_tab, len, 0), "momentum table");
  PIMPC_CHECK(s, cudaDeviceSynchronize(), "momentum table");
  s->coef_len = len;
  return PIMPC_OK;
}

int store_input_sets(pimpc_solver *s, const int *kind, const double *r, const double *a,
                     cudaStream_t st);

void graph_invalidate(pimpc_solver *s) {
  for (auto &g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

int cuda_fail(pimpc_solver *s, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(s, PIMPC_ECUDA, m);
}

size_t tsize(int prec) { return prec == PIMPC_F32 ? 4 : 8; }

cudaError_t dev_in(pimpc_solver *s, const double *p, int64_t count, int mem, int64_t at,
                   cudaStream_t st, const double **out) {
  if (!p) { *out = nullptr; return cudaSuccess; }
  if (mem == PIMPC_DEVICE) { *out = p; return cudaSuccess; }
  double *dst = s->stage64 + at;
  cudaError_t e = cudaMemcpyAsync(dst, p, sizeof(double) * count, cudaMemcpyHostToDevice, st);
  *out = dst;
  return e;
}

}  // namespace pimpc

namespace {

template <typename P>
cudaError_t dalloc(pimpc_solver *s, P **p, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  s->allocs.push_back(q);
  *p = (P *)q;
  return cudaSuccess;
}

bool finite_or_inf_ok(const double *p, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (std::isnan(p[i])) return false;
  return true;
}

}  // namespace


namespace {

void free_layout(pimpc_solver *s) {
  for (void *p : s->lay_allocs) cudaFree(p);
  s->lay_allocs.clear();
  s->blk_T = nullptr;
  for (int b = 0; b < 3; ++b) s->it[b] = nullptr;
  s->item_inst = s->item_a = s->item_b = s->list0 = s->list1 = s->item_first = nullptr;
  s->list_init = s->ccount = s->pos_of = nullptr;
  s->cpart = nullptr;
}

template <typename P>
cudaError_t lalloc(pimpc_solver *s, P **p, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  s->lay_allocs.push_back(q);
  *p = (P *)q;
  return cudaSuccess;
}

}  // namespace

namespace pimpc {

// Lays out the stage blocks and iterates for a schedule, plans the solve kernel's launch and
// work items, and (re)allocates the buffers that depend on them. The iterates restart from zero
// and the factorisation is redone at the next solve.
int apply_schedule(pimpc_solver *s, const Schedule &sc_in, std::string &why) {
  Schedule sc = sc_in;
  const int batch = s->batch, lti = s->lti, precision = s->prec;
  const size_t ts = tsize(precision);
  const std::vector<int> &nx = s->nx, &nu = s->nu, &N = s->N;
  // Default: blocked lane groups for FP32 iterations, plain lane groups for FP64 ones (the FP64
  // pipe bounds those, and the 4-wide padding of the blocked layout adds FP64 work); the other
  // families are chosen explicitly or by the autotuner.
  if (sc.family < 0) sc.family = precision == PIMPC_F32 ? 5 : 0;
  if (sc.family != 0 && sc.family != 2 && sc.family != 3 && sc.family != 4 && sc.family != 5 &&
      sc.family != 6 && sc.family != 7) {
    why = "schedule family must be 0, 2, 3, 4, 5, 6 or 7";
    return PIMPC_EINVAL;
  }
  if (sc.family == 6) {
    if (!lti || precision != PIMPC_F32) {
      why = "the tensor-core schedule serves stage-invariant instances with FP32 iterations";
      return PIMPC_EINVAL;
    }
    for (int j = 0; j < batch; ++j)
      if (!tc_fits(nx[j], nu[j])) {
        why = "the tensor-core schedule needs nx and nu rounded up to 16 to sum to at most 64 "
              "(and nu's to be at most nx's)";
        return PIMPC_EINVAL;
      }
  }
  if (sc.family == 4 && !lti) {
    why = "the contraction schedule serves stage-invariant instances";
    return PIMPC_EINVAL;
  }
  if (sc.family == 2 && (precision != PIMPC_F32 || lti)) {
    why = "halo tiles serve stage-varying FP32 instances";
    return PIMPC_EINVAL;
  }
  if (s->any_uset && sc.family != 0 && sc.family != 5) {
    why = "non-box input sets need schedule family 0 or 5";
    return PIMPC_EINVAL;
  }
  if (sc.ctas_per_sm < 0 || sc.ctas_per_sm > 8 || sc.item_scale < 0 || sc.item_scale > 64) {
    why = "schedule: ctas_per_sm in 0..8, item_scale in 0..64";
    return PIMPC_EINVAL;
  }
  // halo tiles and the blocked lane groups have layouts of their own; the resident and the
  // contraction families read the plain layout
  const int tiled = sc.family == 2 ? 2 : (sc.family == 5 ? 3 : (sc.family == 6 ? 4 : 0));
  s->tiled = tiled;
  int nsm = 0, smem_sm = 0, optin = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
  std::vector<int> W(batch), tw(batch, 0), grp(batch, 0);
  std::vector<int64_t> blk(batch), Ni(batch);
  int64_t tot_blk = 0, tot_Ni = 0;
  AdmmLaunch P{};
  // Items: the coarse ones, then (lane-group families, stage-varying batches) the fine ones of
  // one sub-chunk each, which the solve switches to when few instances are left.
  std::vector<int> item_inst, item_a, item_b, nitems_inst(2 * batch, 0);
  std::vector<int> fine_len(batch, 0);  // stages per fine item (0: no fine items)
  const int fine_sub = 1;                 // sub-chunks per fine item
  const int fine_switch = 1;              // fine items below this many coarse items per CTA
  // Instance order: largest streamed volume first.
  std::vector<int> order(batch);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(batch);
  for (int j = 0; j < batch; ++j) {
    const int n = nx[j] + nu[j];
    cost[j] = (double)N[j] * ((lti ? 0.0 : (double)packed_block_words(nx[j], nu[j])) + 15.0 * n);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  int bps = 0;
  cudaError_t e = cudaSuccess;
  std::vector<int64_t> tc_off(batch, 0);
  int64_t tot_tc = 0;
  if (sc.family == 7) {
    // Windows: per instance the widest window (interior plus T stages on each side) whose shared
    // memory fits the budget of cps CTAs per SM; an instance that fits whole is one closed window.
    const int T = sc.item_scale > 0 ? sc.item_scale : 8;
    const int cps = sc.ctas_per_sm > 0 ? sc.ctas_per_sm : 1;
    const int64_t stat = (int64_t)tb_static_smem(precision);
    const int64_t budget =
        std::min<int64_t>((int64_t)smem_sm / cps - 1024 - stat, optin - stat) / 128 * 128;
    std::vector<int> S(batch), inner(batch);
    for (int j = 0; j < batch; ++j) {
      const int n = nx[j] + nu[j];
      W[j] = block_words(nx[j], nu[j]);
      blk[j] = tot_blk;
      tot_blk += ((int64_t)blocks_per_instance(lti, N[j]) * W[j] + 31) / 32 * 32;
      Ni[j] = tot_Ni;
      tot_Ni += ((int64_t)N[j] * admm_iter_stride(n, precision) + 31) / 32 * 32;
      int lo = 1, hi = N[j];  // the widest window that fits, up to the whole horizon
      if (tb_window_words(nx[j], nu[j], W[j], lti, precision, 1) * (int64_t)ts > budget) lo = 0;
      while (lo > 0 && lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (tb_window_words(nx[j], nu[j], W[j], lti, precision, mid) * (int64_t)ts <= budget) lo = mid;
        else hi = mid - 1;
      }
      S[j] = lo;
      inner[j] = S[j] >= N[j] ? N[j] : S[j] - 2 * T;
      if (inner[j] < 1) {
        char b[200];
        snprintf(b, sizeof b, "instance %d: a window of %d stages leaves no interior at T = %d", j,
                 S[j], T);
        why = b;
        return PIMPC_EINVAL;
      }
      S[j] = std::min(N[j], inner[j] + 2 * T);
    }
    for (int oi = 0; oi < batch; ++oi) {
      const int j = order[oi];
      for (int a0 = 0; a0 < N[j]; a0 += inner[j]) {
        item_inst.push_back(j);
        item_a.push_back(a0);
        item_b.push_back(std::min(N[j], a0 + inner[j]));
        nitems_inst[j] += 1;
      }
    }
    size_t smem = 0;
    for (int j = 0; j < batch; ++j)
      smem = std::max(smem, (size_t)tb_window_words(nx[j], nu[j], W[j], lti, precision, S[j]) * ts);
    s->tb_T = T;
    P.threads = tb_threads();
    s->smem_admm = smem;
    e = tb_configure(precision, smem, &bps);
  } else if (sc.family == 6) {
    // Tiles of 127 stages (128 MMA rows with the stage before the tile); items of a few tiles
    // so that an instance's matrices are copied to shared memory once per item.
    const int tpi = sc.item_scale > 0 ? sc.item_scale : 2;
    size_t smem = 0;
    for (int j = 0; j < batch; ++j) {
      const int n = nx[j] + nu[j];
      W[j] = block_words(nx[j], nu[j]);
      blk[j] = tot_blk;
      tot_blk += ((int64_t)blocks_per_instance(lti, N[j]) * W[j] + 31) / 32 * 32;
      Ni[j] = tot_Ni;
      const int np = ((nx[j] + 15) & ~15) + ((nu[j] + 15) & ~15);
      tot_Ni += ((int64_t)(N[j] + 127) / 128 * 128 * 5 * np + 31) / 32 * 32;
      tc_off[j] = tot_tc;
      tot_tc += tc_block_words(nx[j], nu[j]);
      smem = std::max(smem, tc_smem_bytes(nx[j], nu[j]));
    }
    if (smem + 1024 > (size_t)optin) {
      why = "the tensor-core schedule needs more shared memory than one CTA has";
      return PIMPC_EINVAL;
    }
    for (int oi = 0; oi < batch; ++oi) {
      const int j = order[oi];
      for (int a0 = 0; a0 < N[j]; a0 += 127 * tpi) {
        item_inst.push_back(j);
        item_a.push_back(a0);
        item_b.push_back(std::min(N[j], a0 + 127 * tpi));
        nitems_inst[j] += 1;
      }
    }
    P.threads = tc_threads();
    s->smem_admm = smem;
    e = tc_configure(smem, &bps);
    bps = std::min(bps, 1);
  } else if (sc.family == 4) {
    // Blocks of LB stages (LB from the shared-memory budget of cps CTAs per SM); an item holds
    // several consecutive blocks, so the instance's matrices are expanded once per item.
    const int cps = sc.ctas_per_sm > 0 ? sc.ctas_per_sm : 1;
    int64_t budget = (int64_t)smem_sm / cps - 1024 - 256;
    budget = std::min<int64_t>(budget, optin - 256);
    int mnu = 1;
    for (int j = 0; j < batch; ++j) mnu = std::max(mnu, nu[j]);
    const int LB = gemm_plan(s->max_n, s->max_nx, mnu, precision, (size_t)budget, s->gemm_plan);
    if (LB == 0) {
      why = "the contraction schedule needs more shared memory than the budget";
      return PIMPC_EINVAL;
    }
    const int LBi = sc.item_scale > 0 ? std::min(LB, sc.item_scale) : LB;
    s->gemm_plan[0] = LBi;
    int64_t blocks = 0;
    for (int j = 0; j < batch; ++j) blocks += (N[j] + LBi - 1) / LBi;
    // about four items per SM per iteration, at least one block each
    const int per_item = (int)std::max<int64_t>(1, blocks / (4 * (int64_t)nsm * cps));
    for (int j = 0; j < batch; ++j) {
      const int n = nx[j] + nu[j];
      W[j] = block_words(nx[j], nu[j]);
      blk[j] = tot_blk;
      tot_blk += ((int64_t)blocks_per_instance(lti, N[j]) * W[j] + 31) / 32 * 32;
      Ni[j] = tot_Ni;
      tot_Ni += ((int64_t)N[j] * admm_iter_stride(n, precision) + 31) / 32 * 32;
    }
    for (int oi = 0; oi < batch; ++oi) {
      const int j = order[oi];
      for (int a0 = 0; a0 < N[j]; a0 += LBi * per_item) {
        item_inst.push_back(j);
        item_a.push_back(a0);
        item_b.push_back(std::min(N[j], a0 + LBi * per_item));
        nitems_inst[j] += 1;
      }
    }
    P.threads = gemm_threads();
    s->smem_admm = (size_t)s->gemm_plan[4];
    e = gemm_configure(precision, s->smem_admm, &bps);
  } else if (tiled == 3) {
    // Per instance the most lane groups (S - 1 stages and the next stage per sub-chunk) whose
    // shared memory fits the budget of cps CTAs per SM. By default the cps in 3, 2, 1 with the
    // most stages in flight per SM (cps times the stage-weighted mean of S - 1) among those that
    // fit every instance.
    const int thr = blk_threads();
    auto fit = [&](int cps, std::vector<int> &S_of, int64_t &bud) {
      bud = std::min<int64_t>((int64_t)smem_sm / cps - 1024 - 256, optin - 256) / 128 * 128;
      for (int j = 0; j < batch; ++j) {
        int S = thr / bl_group(nx[j] + nu[j]);
        while (S >= 2 && blk_region_words(nx[j], nu[j], lti, precision, S) * (int64_t)ts > bud) --S;
        if (S < 2) return j;
        S_of[j] = S;
      }
      return -1;
    };
    int64_t budget = 0;
    int bad = -1;
    if (sc.ctas_per_sm > 0) {
      bad = fit(sc.ctas_per_sm, grp, budget);
    } else {
      double best = -1.0;
      std::vector<int> S_try(batch);
      for (int cps = 3; cps >= 1; --cps) {
        int64_t b = 0;
        const int r = fit(cps, S_try, b);
        if (r >= 0) { if (best < 0.0) { bad = r; budget = b; } continue; }
        double num = 0.0, den = 0.0;
        for (int j = 0; j < batch; ++j) {
          num += (double)N[j] * (S_try[j] - 1);
          den += (double)N[j];
        }
        const double score = cps * num / den;
        if (score > best) { best = score; grp = S_try; budget = b; bad = -1; }
      }
    }
    if (bad >= 0) {
      char b[200];
      snprintf(b, sizeof b, "instance %d (nx %d, nu %d) does not fit the blocked schedule in %lld bytes",
               bad, nx[bad], nu[bad], (long long)budget);
      why = b;
      return PIMPC_EINVAL;
    }
    int64_t words_max = 4, total_sub = 0;
    for (int j = 0; j < batch; ++j) {
      const int n = nx[j] + nu[j];
      const int S = grp[j];
      words_max = std::max<int64_t>(words_max, blk_region_words(nx[j], nu[j], lti, precision, S));
      W[j] = bl_block_words(nx[j], nu[j], (int)ts);
      blk[j] = tot_blk;
      tot_blk += ((int64_t)blocks_per_instance(lti, N[j]) * W[j] + 31) / 32 * 32;
      Ni[j] = tot_Ni;
      tot_Ni += ((int64_t)N[j] * bl_rec(n) + 31) / 32 * 32;
      total_sub += (N[j] + S - 2) / (S - 1);
    }
    P.threads = thr;
    s->smem_admm = (size_t)words_max * ts;
    e = blk_configure(precision, s->smem_admm, &bps);
    if (e == cudaSuccess && bps >= 1) {
      const int64_t max_grid = (int64_t)bps * nsm;
      // Sub-chunks per item: enough items for about 4 per CTA, at most 64 sub-chunks per item.
      int64_t m = sc.item_scale > 0 ? sc.item_scale : total_sub / (4 * max_grid);
      m = std::max<int64_t>(1, std::min<int64_t>(64, m));
      for (int oi = 0; oi < batch; ++oi) {
        const int j = order[oi];
        const int P1 = grp[j] - 1;
        int is = (int)(P1 * m);
        if (lti) is = std::max(is, std::min(N[j], (256 + P1 - 1) / P1 * P1));
        if (!lti && m > fine_sub) fine_len[j] = P1 * fine_sub;
        for (int a0 = 0; a0 < N[j]; a0 += is) {
          item_inst.push_back(j);
          item_a.push_back(a0);
          item_b.push_back(std::min(N[j], a0 + is));
          nitems_inst[j] += 1;
        }
      }
    }
  } else if (tiled == 2) {
    // Shared-memory budget of one CTA, and per instance the widest tile that fits it.
    const int cps = sc.ctas_per_sm > 0 ? sc.ctas_per_sm : 2;
    int64_t D = (int64_t)smem_sm / cps - 1024 - 256;
    D = std::min<int64_t>(D, optin - 256);
    D = D / 128 * 128;
    const int max_tiles = sc.item_scale > 0 ? std::min(sc.item_scale, tile_warps()) : tile_warps();
    auto tile_bytes = [&](int j, int w) {
      const int n = nx[j] + nu[j];
      return (int64_t)(tile_block_words(w, nx[j], nu[j]) + 2 * tile_iter_words(w, n) + 4 * n * w) *
             (int64_t)ts;
    };
    for (int j = 0; j < batch; ++j) {
      const int n = nx[j] + nu[j];
      int w = 0;
      for (int cand : {32, 16})
        if (tile_bytes(j, cand) <= D) { w = cand; break; }
      if (w == 0) {
        char b[200];
        snprintf(b, sizeof b, "instance %d (nx %d, nu %d) does not fit a halo tile in %lld bytes",
                 j, nx[j], nu[j], (long long)D);
        why = b;
        return PIMPC_EINVAL;
      }
      tw[j] = w;
      const int nt = halo_tiles(N[j], w);
      W[j] = tile_block_words(w, nx[j], nu[j]);
      blk[j] = tot_blk;
      tot_blk += ((int64_t)nt * W[j] + 31) / 32 * 32;
      Ni[j] = tot_Ni;
      tot_Ni += ((int64_t)nt * tile_iter_words(w, n) + 31) / 32 * 32;
    }
    for (int oi = 0; oi < batch; ++oi) {
      const int j = order[oi];
      const int nt = halo_tiles(N[j], tw[j]);
      const int m = (int)std::max<int64_t>(1, std::min<int64_t>(max_tiles, D / tile_bytes(j, tw[j])));
      for (int t0 = 0; t0 < nt; t0 += m) {
        item_inst.push_back(j);
        item_a.push_back(t0);
        item_b.push_back(std::min(nt, t0 + m));
        nitems_inst[j] += 1;
      }
    }
    P.threads = tile_threads();
    P.capB = (int)(D / (int64_t)ts);
    s->smem_admm = (size_t)D;
    e = tile_configure(s->smem_admm, &bps);
  } else {
    const int threads = admm_threads(precision);
    int nv_max = 2, W_max = 4, n5p_max = 4, scr_max = 4, xrows_max = 4;
    int64_t capB = 0, capI = 0, total_sub = 0;
    for (int j = 0; j < batch; ++j) {
      const int n = nx[j] + nu[j];
      const int n5p = admm_iter_stride(n, precision);
      W[j] = block_words(nx[j], nu[j]);
      blk[j] = tot_blk;
      tot_blk += ((int64_t)blocks_per_instance(lti, N[j]) * W[j] + 31) / 32 * 32;
      Ni[j] = tot_Ni;
      tot_Ni += ((int64_t)N[j] * n5p + 31) / 32 * 32;
      const int S = threads / admm_group_size(n);
      const int nv = (n + 3) & ~3;
      scr_max = std::max(scr_max, S * 4 * nv);            // per-group scratch rows
      xrows_max = std::max(xrows_max, 2 * (S + 1) * nv);  // double-buffered xbar rows
      nv_max = std::max(nv_max, nv);
      W_max = std::max(W_max, W[j]);
      n5p_max = std::max(n5p_max, n5p);
      if (!lti) {
        // S stage blocks plus the next stage's G and e (see the solve kernel's copies)
        const int ge = (nx[j] * odd_ld(n) + nx[j] + 3) & ~3;
        capB = std::max<int64_t>(capB, (int64_t)S * W[j] + ge);
      }
      capI = std::max<int64_t>(capI, (int64_t)(S + 1) * n5p);
      total_sub += (N[j] + S - 1) / S;
    }
    P.threads = threads;
    P.capB = (int)capB;
    P.capI = (int)capI;
    P.haloB = lti ? 2 * W_max : W_max;
    P.haloI = 2 * n5p_max;
    P.S_max = scr_max;    // the lane-group kernel's plan takes the scratch and xbar-row sizes
    P.nv_max = xrows_max;
    P.nbuf = 1;
    s->smem_admm = admm_smem_bytes(P, precision);
    if (s->smem_admm + 1024 > (size_t)optin) {
      why = "an instance needs more shared memory than one CTA has at this precision";
      return PIMPC_EINVAL;
    }
    e = admm_configure(precision, s->smem_admm, &bps);
    if (sc.family == 3 && e == cudaSuccess) {
      // One CTA or a cluster per instance: the fewest CTAs whose shared memory holds a slice.
      const int thr = res_threads(precision);
      int plan[6];
      size_t bytes = 0;
      int C = 0;
      // With item_scale = 0: the fewest CTAs that fit, or, when the whole batch occupies few
      // SMs (latency, not throughput, is what a small batch needs), the most CTAs (up to 16)
      // that still give every CTA four stages or more.
      const int nmin = *std::min_element(N.begin(), N.end());
      int fewest = 0, most = 0;
      size_t b_few = 0, b_most = 0;
      int p_few[6], p_most[6];
      for (int cand : {1, 2, 4, 8, 16}) {
        if (sc.item_scale > 0 && cand != sc.item_scale) continue;
        const size_t b = res_plan(batch, nx.data(), nu.data(), N.data(), W.data(), lti, precision,
                                  thr, cand, plan);
        if (b == 0 || b + 1024 > (size_t)optin - 256) continue;
        if (fewest == 0) { fewest = cand; b_few = b; std::copy(plan, plan + 6, p_few); }
        if (sc.item_scale > 0 || (nmin >= 4 * cand && (int64_t)batch * cand <= nsm)) {
          most = cand; b_most = b; std::copy(plan, plan + 6, p_most);
        }
      }
      if (most > 0 && most >= fewest) {
        C = most; bytes = b_most; std::copy(p_most, p_most + 6, plan);
      } else if (fewest > 0) {
        C = fewest; bytes = b_few; std::copy(p_few, p_few + 6, plan);
      }
      if (C == 0) {
        why = "the instances do not fit the shared memory of a cluster of that size (or N < cluster size)";
        return PIMPC_EINVAL;
      }
      std::copy(plan, plan + 6, s->res_plan);
      P.threads = thr;
      s->smem_admm = bytes;
    }
    if (e == cudaSuccess && bps >= 1) {
      const int64_t max_grid = (int64_t)bps * nsm;
      // Sub-chunks per item: enough items for about 4 per CTA, at most 16 sub-chunks per item.
      int64_t m = sc.item_scale > 0 ? sc.item_scale : total_sub / (4 * max_grid);
      m = std::max<int64_t>(1, std::min<int64_t>(sc.item_scale > 0 ? 64 : 16, m));
      for (int oi = 0; oi < batch; ++oi) {
        const int j = order[oi];
        const int n = nx[j] + nu[j];
        const int S = threads / admm_group_size(n);
        int is = (int)(S * m);
        if (lti) is = std::max(is, std::min(N[j], (256 + S - 1) / S * S));
        if (!lti && m > fine_sub) fine_len[j] = S * fine_sub;
        for (int a0 = 0; a0 < N[j]; a0 += is) {
          item_inst.push_back(j);
          item_a.push_back(a0);
          item_b.push_back(std::min(N[j], a0 + is));
          nitems_inst[j] += 1;
        }
      }
    }
  }
  if (e != cudaSuccess || bps < 1) {
    why = std::string("kernel configuration failed: ") +
          (e != cudaSuccess ? cudaGetErrorString(e) : "zero occupancy");
    return PIMPC_ECUDA;
  }
  const int nitems = (int)item_inst.size();
  const int grid = (int)std::min<int64_t>((int64_t)bps * nsm, nitems);
  for (int oi = 0; oi < batch; ++oi) {
    const int j = order[oi];
    if (fine_len[j] <= 0) continue;
    for (int a0 = 0; a0 < N[j]; a0 += fine_len[j]) {
      item_inst.push_back(j);
      item_a.push_back(a0);
      item_b.push_back(std::min(N[j], a0 + fine_len[j]));
      nitems_inst[batch + j] += 1;
    }
  }
  const int nall = (int)item_inst.size();
  // The items of an instance are consecutive (coarse ones, then fine ones): the per-iteration
  // finish pass sums an instance's shares of c over [first, first + count).
  std::vector<int> item_first(2 * batch, 0);
  for (int i = nall - 1; i >= 0; --i) item_first[item_inst[i] + (i >= nitems ? batch : 0)] = i;
  for (int i = 0; i < nall; ++i) {
    const int j = item_inst[i], f = i >= nitems ? batch : 0;
    if (i >= item_first[j + f] + nitems_inst[j + f]) {
      why = "internal: the items of an instance are not consecutive";
      return PIMPC_EINVAL;
    }
  }
  // The active list starts with the coarse items longest first (streamed volume), so that the
  // queue hands out the long items first and the short ones fill the end of the iteration.
  std::vector<int> list_init(nitems);
  std::iota(list_init.begin(), list_init.end(), 0);
  {
    std::vector<double> icost(nitems);
    for (int i = 0; i < nitems; ++i) {
      const int j = item_inst[i];
      icost[i] = cost[j] / (double)N[j] * (double)(item_b[i] - item_a[i]);
    }
    std::stable_sort(list_init.begin(), list_init.end(),
                     [&](int x, int y) { return icost[x] > icost[y]; });
  }

  // (Re)allocate and upload what depends on the schedule.
  cudaDeviceSynchronize();
  graph_invalidate(s);
  free_layout(s);
  e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  int64_t *d_blk = nullptr, *d_Ni = nullptr;
  int *d_W = nullptr, *d_tw = nullptr, *d_grp = nullptr;
  chk(lalloc(s, &s->blk_T, ts * tot_blk));
  for (int b = 0; b < 3; ++b) chk(lalloc(s, &s->it[b], ts * tot_Ni));
  chk(lalloc(s, &s->item_inst, sizeof(int) * nall));
  chk(lalloc(s, &s->item_a, sizeof(int) * nall));
  chk(lalloc(s, &s->item_b, sizeof(int) * nall));
  chk(lalloc(s, &s->list0, sizeof(int) * nall));
  chk(lalloc(s, &s->list1, sizeof(int) * nall));
  chk(lalloc(s, &s->item_first, sizeof(int) * 2 * batch));
  chk(lalloc(s, &s->cpart, sizeof(double) * nall));
  chk(lalloc(s, &s->list_init, sizeof(int) * std::max(nitems, 1)));
  chk(lalloc(s, &s->ccount, sizeof(int) * std::max(grid, 1)));
  chk(lalloc(s, &s->pos_of, sizeof(int) * nall));
  chk(lalloc(s, &d_blk, sizeof(int64_t) * batch));
  chk(lalloc(s, &d_Ni, sizeof(int64_t) * batch));
  chk(lalloc(s, &d_W, sizeof(int) * batch));
  chk(lalloc(s, &d_tw, sizeof(int) * batch));
  chk(lalloc(s, &d_grp, sizeof(int) * batch));
  s->tc_mat = nullptr;
  s->tc_off = nullptr;
  if (sc.family == 6) {
    chk(lalloc(s, &s->tc_mat, sizeof(float) * (size_t)tot_tc));
    chk(lalloc(s, &s->tc_off, sizeof(int64_t) * batch));
  }
  if (e != cudaSuccess) {
    why = std::string("device allocation failed: ") + cudaGetErrorString(e);
    const bool oom = e == cudaErrorMemoryAllocation;
    free_layout(s);
    (void)cudaGetLastError();
    return oom ? PIMPC_ENOMEM : PIMPC_ECUDA;
  }
  chk(cudaMemcpy(s->item_inst, item_inst.data(), sizeof(int) * nall, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(s->item_a, item_a.data(), sizeof(int) * nall, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(s->item_b, item_b.data(), sizeof(int) * nall, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(s->nitems_inst, nitems_inst.data(), sizeof(int) * 2 * batch, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(s->item_first, item_first.data(), sizeof(int) * 2 * batch, cudaMemcpyHostToDevice));
  chk(cudaMemset(s->cpart, 0, sizeof(double) * nall));
  chk(cudaMemcpy(s->list_init, list_init.data(), sizeof(int) * nitems, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(d_blk, blk.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(d_Ni, Ni.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(d_W, W.data(), sizeof(int) * batch, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(d_tw, tw.data(), sizeof(int) * batch, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(d_grp, grp.data(), sizeof(int) * batch, cudaMemcpyHostToDevice));
  if (sc.family == 6)
    chk(cudaMemcpy(s->tc_off, tc_off.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice));
  chk(cudaMemset(s->blk_T, 0, ts * tot_blk));
  for (int b = 0; b < 3; ++b) chk(cudaMemset(s->it[b], 0, ts * tot_Ni));
  chk(cudaMemset(s->base, 0, sizeof(int) * batch));
  chk(cudaDeviceSynchronize());
  if (e != cudaSuccess) {
    why = std::string("device initialisation failed: ") + cudaGetErrorString(e);
    free_layout(s);
    return PIMPC_ECUDA;
  }
  s->W = W;
  s->tw = tw;
  s->blk = blk;
  s->Ni = Ni;
  s->tot_blk = tot_blk;
  s->tot_Ni = tot_Ni;
  s->nitems = nitems;
  s->grid_admm = grid;
  P.grid = grid;
  P.grp = d_grp;
  P.nfine_base = nitems;
  P.nfine = nall - nitems;
  P.fine_switch = fine_switch;
  s->plan = P;
  s->sched = sc;
  s->L.tiled = tiled;
  s->L.tw = tiled == 2 ? d_tw : nullptr;
  s->L.blk = d_blk;
  s->L.Ni = d_Ni;
  s->L.W = d_W;
  s->stale = true;
  s->solved = false;
  return ensure_coef_table(s);
}

}  // namespace pimpc

namespace {

// One solve on FP64 device inputs: the stage cache if stale, xbar_0 and the reference in the
// iteration precision, then the persistent launch; u_dev, x_dev (device, may be null) receive
// the outputs.
int run_solve(pimpc_solver *s, const double *dx0, const double *dup, const double *dref,
              int ref_per_stage, int warm_start, double *u_dev, double *x_dev, cudaStream_t st) {
  if (s->stale) {
    const int rc = pimpc_factorise(s, st);
    if (rc) return rc;
  }
  if (!s->solved) warm_start = 0;  // nothing to reuse after a new schedule
  const int64_t nref = ref_per_stage ? s->tot_Nn : s->tot_n;
  PIMPC_CHECK(s, launch_gather_n(s->L, dx0, dup, s->tot_n, s->prec, s->xb0_T, st), "x0");
  if (dref) PIMPC_CHECK(s, launch_convert(dref, nref, s->prec, s->ref_T, st), "ref");
  AdmmLaunch a = s->plan;
  a.L = s->L; a.blk = s->blk_T;
  for (int b = 0; b < 3; ++b) a.it[b] = s->it[b];
  a.qd = s->qd_T; a.ref = dref ? s->ref_T : nullptr; a.ref_per_stage = ref_per_stage;
  a.lo = s->lo_T; a.hi = s->hi_T; a.xb0 = s->xb0_T;
  a.rho = s->rho; a.eps = s->eps; a.eta = s->eta; a.max_iters = s->max_iters; a.accel = s->accel;
  a.mask = s->mask; a.mask_len = s->mask_len;
  a.item_inst = s->item_inst; a.item_a = s->item_a; a.item_b = s->item_b;
  a.nitems_inst = s->nitems_inst; a.nitems = s->nitems;
  a.item_first = s->item_first; a.cpart = s->cpart;
  a.list_init = s->list_init; a.ccount = s->ccount; a.pos_of = s->pos_of;
  a.list0 = s->list0; a.list1 = s->list1; a.ctl = s->ctl;
  a.base = s->base; a.old_base = s->old_base; a.st = s->st;
  a.alpha = s->alpha; a.cprev = s->cprev; a.coef = s->coef; a.cacc = s->cacc;
  a.ndone = s->ndone; a.stop = s->stop;
  a.warm = warm_start;
  a.ferr = s->ferr;
  a.bar_limit = s->bar_limit;
  a.stall_win = s->stall_win;
  a.uset_kind = s->any_uset ? s->uset_kind_d : nullptr;
  a.uset_r = s->any_uset ? s->uset_r_T : nullptr;
  a.uset_a = s->any_uset ? s->uset_a_T : nullptr;
  a.stall_fac = s->stall_fac;
  a.stall_below = s->stall_below;
  a.stall_rel = s->stall_rel;
  a.itfirst = s->itfirst;
  a.cbest = s->cbest;
  a.itbest = s->itbest;
  a.u_out = u_dev;
  a.x_out = x_dev;
  a.coef_tab = s->coef_tab;
  if (s->sched.family == 3 && s->coef_len < s->max_iters + 1)
    return fail(s, PIMPC_ESTATE, "momentum table shorter than max_iters");
  if (s->sched.family == 7 && s->accel)
    return fail(s, PIMPC_ESTATE, "temporal blocking (schedule 7) runs the plain iteration: accel must be 0");
  PIMPC_CHECK(s, s->tiled == 2 ? launch_tile(a, st)
                 : s->tiled == 3 ? launch_blk(a, s->prec, s->smem_admm, st)
                 : s->sched.family == 3 ? launch_resident(a, s->prec, s->res_plan, s->smem_admm, st)
                 : s->sched.family == 4 ? launch_gemm(a, s->prec, s->gemm_plan, st)
                 : s->sched.family == 6 ? launch_tc(a, s->tc_mat, s->tc_off, s->smem_admm, st)
                 : s->sched.family == 7 ? launch_tb(a, s->prec, s->tb_T, s->smem_admm, st)
                                        : launch_admm(a, s->prec, st),
              "solve");
  s->solved = true;
  s->last_ref_per_stage = ref_per_stage;
  s->last_ref_given = dref != nullptr;
  s->last_warm = warm_start;
  s->last_accel = s->accel;
  s->last_eps = s->eps;
  s->last_iters_fixed = s->max_iters;
  return PIMPC_OK;
}

// FP64 polish after an FP32 solve: FP64 iterations (the FP64 stage cache, FP64 residual c)
// started from the FP32 iterates, run by an FP64 solver object that reads this solver's FP64
// dynamics, weights and bounds. Per-instance results become the sum of both iteration counts
// and the polish's c and status.
// Host-side and eager part of the polish: the FP64 solver, its options, weights, bounds and (if
// the inputs changed) its stage cache.
int prepare_polish(pimpc_solver *s, cudaStream_t st) {
  if (!s->shadow) {
    pimpc_solver *sh = nullptr;
    const int rc = pimpc_create(s->batch, s->nx.data(), s->nu.data(), s->N.data(), s->lti,
                                PIMPC_F64, s->device, &sh);
    if (rc != PIMPC_OK) return fail(s, rc, std::string("polish solver: ") + pimpc_last_error(nullptr));
    s->shadow = sh;
    s->shadow_fgen = -1;
  }
  pimpc_solver *sh = s->shadow;
  sh->rho = s->rho;
  sh->eps = s->polish_eps;
  sh->max_iters = s->polish_iters;
  sh->accel = s->accel;
  sh->eta = s->eta;
  const size_t nb = sizeof(double) * s->tot_n;
  PIMPC_CHECK(s, cudaMemcpyAsync(sh->qd_T, s->qd64, nb, cudaMemcpyDeviceToDevice, st), "polish weights");
  PIMPC_CHECK(s, cudaMemcpyAsync(sh->lo_T, s->lo64, nb, cudaMemcpyDeviceToDevice, st), "polish bounds");
  PIMPC_CHECK(s, cudaMemcpyAsync(sh->hi_T, s->hi64, nb, cudaMemcpyDeviceToDevice, st), "polish bounds");
  if (s->shadow_fgen != s->fgen) {
    PIMPC_CHECK(s, launch_factorise(sh->L, s->A64, s->B64, s->e64, s->qd64,
                                    s->have_rdu ? s->rdu64 : nullptr, s->rho, sh->binst,
                                    sh->d_bbase, sh->nblocks, sh->max_nx, sh->max_n, PIMPC_F64,
                                    sh->blk_T, sh->ferr, st),
                "polish factorise");
    s->shadow_fgen = s->fgen;
  }
  if (s->any_uset != sh->any_uset || s->any_uset) {
    const int rc = store_input_sets(sh, s->uset_kind_h.data(), s->uset_r_h.data(),
                                    s->uset_a_h.data(), st);
    if (rc != PIMPC_OK) return fail(s, rc, std::string("polish input sets: ") + sh->err);
  }
  sh->stale = false;
  sh->solved = true;
  return PIMPC_OK;
}

// The launches of the polish (capturable): FP32 iterates -> FP64 start, FP64 solve, results.
int polish_launch(pimpc_solver *s, const double *dx0, const double *dup, const double *dref,
                  int ref_per_stage, double *u_dev, double *x_dev, cudaStream_t st) {
  pimpc_solver *sh = s->shadow;
  PIMPC_CHECK(s, launch_copy_iterates(s->L, s->it, s->base, s->prec, sh->L, sh->it, sh->base, st),
              "polish start");
  const int rc = run_solve(sh, dx0, dup, dref, ref_per_stage, 1, u_dev, x_dev, st);
  if (rc != PIMPC_OK) return fail(s, rc, std::string("polish: ") + sh->err);
  PIMPC_CHECK(s, launch_add_state(s->st, sh->st, s->batch, st), "polish state");
  return PIMPC_OK;
}

// Device-memory solve through a CUDA graph: the launches of one solve (x0 and reference
// conversion, the per-instance reset, the starting iterates, the persistent cooperative kernel,
// the outputs, the polish and the status unpacking) are captured once per argument set and
// replayed by later calls with the same arguments; the stage cache (when stale) and the
// polish's host-side preparation run before, outside the graph. A refused capture sets
// graph_failed and leaves the caller to run the launches directly.
int graph_solve(pimpc_solver *s, const double *dx0, const double *dup, const double *dref,
                int ref_per_stage, int warm_start, double *u_dev, double *x_dev, int *iters,
                double *c, int *status, bool polish, cudaStream_t st) {
  if (s->stale) {
    const int rc = pimpc_factorise(s, st);
    if (rc) return rc;
  }
  if (polish) {
    const int rc = prepare_polish(s, st);
    if (rc) return rc;
  }
  const int warm = s->solved ? warm_start : 0;
  const std::vector<uintptr_t> key = {
      (uintptr_t)dx0, (uintptr_t)dup, (uintptr_t)dref, (uintptr_t)ref_per_stage, (uintptr_t)warm,
      (uintptr_t)u_dev, (uintptr_t)x_dev, (uintptr_t)iters, (uintptr_t)c, (uintptr_t)status,
      (uintptr_t)polish};
  pimpc_solver::GraphEntry *hit = nullptr;
  for (auto &g : s->graphs)
    if (g.key == key) hit = &g;
  if (!hit) {
    if (!s->cap_stream) PIMPC_CHECK(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = PIMPC_OK;
    if (e == cudaSuccess) {
      rc = run_solve(s, dx0, dup, dref, ref_per_stage, warm, polish ? nullptr : u_dev,
                     polish ? nullptr : x_dev, s->cap_stream);
      if (rc == PIMPC_OK && polish)
        rc = polish_launch(s, dx0, dup, dref, ref_per_stage, u_dev, x_dev, s->cap_stream);
      if (rc == PIMPC_OK && (iters || c || status)) {
        const cudaError_t e3 = launch_unpack_state(s->st, s->batch, iters, c, status, nullptr, s->cap_stream);
        if (e3 != cudaSuccess) rc = cuda_fail(s, e3, "state");
      }
      const cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && rc == PIMPC_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || rc != PIMPC_OK) {
      s->graph_failed = 1;
      s->graph_err = e != cudaSuccess ? cudaGetErrorString(e) : s->err;
      (void)cudaGetLastError();
      return PIMPC_OK;
    }
    if (s->graphs.size() >= 8) {
      cudaGraphExecDestroy(s->graphs.front().exec);
      s->graphs.erase(s->graphs.begin());
    }
    s->graphs.push_back({key, exec, warm, ref_per_stage, dref != nullptr, polish ? 1 : 0});
    hit = &s->graphs.back();
    ++s->graph_captures;
  } else {
    ++s->graph_replays;
  }
  PIMPC_CHECK(s, cudaGraphLaunch(hit->exec, st), "graph launch");
  s->solved = true;
  s->last_ref_per_stage = hit->ref_per_stage;
  s->last_ref_given = hit->ref_given;
  s->last_warm = hit->warm;
  s->last_accel = s->accel;
  s->last_eps = s->eps;
  s->last_iters_fixed = s->max_iters;
  s->last_polished = hit->polished != 0;
  return PIMPC_OK;
}

}  // namespace

extern "C" {

const char *pimpc_last_error(const pimpc_solver *s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

void pimpc_destroy(pimpc_solver *s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (void *p : s->allocs) cudaFree(p);
  for (void *p : s->lay_allocs) cudaFree(p);
  if (s->adj_ws) cudaFree(s->adj_ws);
  if (s->shadow) pimpc_destroy(s->shadow);
  if (s->coef_tab) cudaFree(s->coef_tab);
  graph_invalidate(s);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->mask_alloc) cudaFree(s->mask_alloc);
  if (s->uset_kind_d) cudaFree(s->uset_kind_d);
  if (s->uset_r_T) cudaFree(s->uset_r_T);
  if (s->uset_a_T) cudaFree(s->uset_a_T);
  delete s;
}

int pimpc_create(int batch, const int *nx, const int *nu, const int *N, int lti, int precision,
                 int device, pimpc_solver **out) {
  if (!out) { g_create_error = "out is NULL"; return PIMPC_EINVAL; }
  *out = nullptr;
  if (batch < 1 || !nx || !nu || !N) { g_create_error = "batch < 1 or NULL size arrays"; return PIMPC_EINVAL; }
  if (precision != PIMPC_F32 && precision != PIMPC_F64) { g_create_error = "bad precision"; return PIMPC_EINVAL; }
  if (lti != 0 && lti != 1) { g_create_error = "lti must be 0 or 1"; return PIMPC_EINVAL; }
  const int nmax = lti ? PIMPC_MAX_N_LTI : PIMPC_MAX_N_LTV;
  for (int j = 0; j < batch; ++j) {
    if (nx[j] < 1 || nu[j] < 1 || N[j] < 1 || nx[j] + nu[j] > nmax || nu[j] > PIMPC_MAX_NU) {
      char b[200];
      snprintf(b, sizeof b,
               "instance %d: need nx >= 1, 1 <= nu <= %d, N >= 1, nx + nu <= %d (got %d, %d, %d)",
               j, PIMPC_MAX_NU, nmax, nx[j], nu[j], N[j]);
      g_create_error = b;
      return PIMPC_EINVAL;
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    g_create_error = "no such CUDA device";
    return PIMPC_ECUDA;
  }
  cudaSetDevice(device);
  pimpc_solver *s = new pimpc_solver();
  s->device = device; s->batch = batch; s->lti = lti; s->prec = precision;
  s->nx.assign(nx, nx + batch); s->nu.assign(nu, nu + batch); s->N.assign(N, N + batch);
  auto grow = [&](std::vector<int64_t> &v, int64_t &tot, int64_t add) { v.push_back(tot); tot += add; };
  const size_t ts = tsize(precision);
  int64_t stage_acc = 0;
  for (int j = 0; j < batch; ++j) {
    const int n = nx[j] + nu[j];
    grow(s->off_nx, s->tot_nx, nx[j]);
    grow(s->off_nu, s->tot_nu, nu[j]);
    grow(s->off_n, s->tot_n, n);
    grow(s->Nnx, s->tot_Nnx, (int64_t)N[j] * nx[j]);
    grow(s->Nnu, s->tot_Nnu, (int64_t)N[j] * nu[j]);
    grow(s->Nn, s->tot_Nn, (int64_t)N[j] * n);
    const int64_t reps = lti ? 1 : N[j];
    grow(s->offA, s->tot_A, reps * nx[j] * nx[j]);
    grow(s->offB, s->tot_B, reps * nx[j] * nu[j]);
    grow(s->offe, s->tot_e, reps * nx[j]);
    s->stage0.push_back(stage_acc);
    stage_acc += N[j];
    grow(s->bbase, s->nblocks, blocks_per_instance(lti, N[j]));
    s->max_nx = std::max(s->max_nx, nx[j]);
    s->max_n = std::max(s->max_n, n);
  }
  std::vector<int> binst(s->nblocks);
  for (int j = 0; j < batch; ++j)
    for (int b = 0; b < blocks_per_instance(lti, N[j]); ++b) binst[s->bbase[j] + b] = j;

  const int64_t stage_words = std::max<int64_t>(
      {2 * s->tot_nx + 2 * s->tot_nu, s->tot_nx + s->tot_nu + s->tot_Nn,
       s->tot_Nnx + s->tot_Nnu + 8 * (int64_t)batch, s->tot_Nnx + s->tot_Nnu + 2 * s->tot_Nn,
       s->tot_n + s->tot_Nn});
  s->stage_words = stage_words;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  std::vector<int64_t> *h_off[10] = {&s->off_nx, &s->off_nu, &s->off_n, &s->Nnx, &s->Nnu, &s->Nn,
                                     &s->offA, &s->offB, &s->offe, &s->stage0};
  int64_t *d_off[10];
  for (int i = 0; i < 10; ++i) {
    chk(dalloc(s, &d_off[i], sizeof(int64_t) * batch));
    if (e == cudaSuccess) chk(cudaMemcpy(d_off[i], h_off[i]->data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice));
  }
  int *d_nx = nullptr, *d_nu = nullptr, *d_N = nullptr;
  chk(dalloc(s, &d_nx, sizeof(int) * batch));
  chk(dalloc(s, &d_nu, sizeof(int) * batch));
  chk(dalloc(s, &d_N, sizeof(int) * batch));
  chk(dalloc(s, &s->d_bbase, sizeof(int64_t) * batch));
  if (e == cudaSuccess) {
    chk(cudaMemcpy(d_nx, nx, sizeof(int) * batch, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(d_nu, nu, sizeof(int) * batch, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(d_N, N, sizeof(int) * batch, cudaMemcpyHostToDevice));
    chk(cudaMemcpy(s->d_bbase, s->bbase.data(), sizeof(int64_t) * batch, cudaMemcpyHostToDevice));
  }
  chk(dalloc(s, &s->A64, sizeof(double) * s->tot_A));
  chk(dalloc(s, &s->B64, sizeof(double) * s->tot_B));
  chk(dalloc(s, &s->e64, sizeof(double) * s->tot_e));
  chk(dalloc(s, &s->qd64, sizeof(double) * s->tot_n));
  chk(dalloc(s, &s->rdu64, sizeof(double) * s->tot_n));
  chk(dalloc(s, &s->stage64, sizeof(double) * stage_words));
  chk(dalloc(s, &s->out_u, sizeof(double) * s->tot_Nnu));
  chk(dalloc(s, &s->out_x, sizeof(double) * s->tot_Nnx));
  chk(dalloc(s, &s->qd_T, ts * s->tot_n));
  chk(dalloc(s, &s->ref_T, ts * std::max(s->tot_Nn, s->tot_n)));
  chk(dalloc(s, &s->lo_T, ts * s->tot_n));
  chk(dalloc(s, &s->hi_T, ts * s->tot_n));
  chk(dalloc(s, &s->xb0_T, ts * s->tot_n));
  chk(dalloc(s, &s->lo64, sizeof(double) * s->tot_n));
  chk(dalloc(s, &s->hi64, sizeof(double) * s->tot_n));
  chk(dalloc(s, &s->base, sizeof(int) * batch));
  chk(dalloc(s, &s->old_base, sizeof(int) * batch));
  chk(dalloc(s, &s->alpha, sizeof(double) * batch));
  chk(dalloc(s, &s->cprev, sizeof(double) * batch));
  chk(dalloc(s, &s->coef, sizeof(double) * batch));
  chk(dalloc(s, &s->cacc, sizeof(double) * batch));
  chk(dalloc(s, &s->cbest, sizeof(double) * batch));
  chk(dalloc(s, &s->itbest, sizeof(int) * batch));
  chk(dalloc(s, &s->itfirst, sizeof(int) * batch));
  chk(dalloc(s, &s->ndone, sizeof(int) * batch));
  chk(dalloc(s, &s->stop, sizeof(int) * batch));
  chk(dalloc(s, &s->nitems_inst, sizeof(int) * 2 * batch));
  chk(dalloc(s, &s->ctl, sizeof(Ctl)));
  chk(dalloc(s, &s->binst, sizeof(int) * s->nblocks));
  chk(dalloc(s, &s->ferr, sizeof(int) * (size_t)batch));
  chk(dalloc(s, &s->st, sizeof(InstState) * batch));
  if (e != cudaSuccess) {
    g_create_error = std::string("device allocation failed: ") + cudaGetErrorString(e);
    const bool oom = e == cudaErrorMemoryAllocation;
    pimpc_destroy(s);
    return oom ? PIMPC_ENOMEM : PIMPC_ECUDA;
  }
  chk(cudaMemcpy(s->binst, binst.data(), sizeof(int) * s->nblocks, cudaMemcpyHostToDevice));
  chk(cudaMemset(s->A64, 0, sizeof(double) * s->tot_A));
  chk(cudaMemset(s->B64, 0, sizeof(double) * s->tot_B));
  chk(cudaMemset(s->e64, 0, sizeof(double) * s->tot_e));
  chk(cudaMemset(s->qd64, 0, sizeof(double) * s->tot_n));
  chk(cudaMemset(s->rdu64, 0, sizeof(double) * s->tot_n));
  chk(cudaMemset(s->qd_T, 0, ts * s->tot_n));
  chk(cudaMemset(s->ferr, 0, sizeof(int) * (size_t)batch));
  chk(cudaMemset(s->st, 0, sizeof(InstState) * batch));
  {
    std::vector<double> inf(s->tot_n, INFINITY);
    chk(cudaMemcpy(s->hi64, inf.data(), sizeof(double) * s->tot_n, cudaMemcpyHostToDevice));
    chk(launch_convert(s->hi64, s->tot_n, precision, s->hi_T, 0));
    for (auto &v : inf) v = -INFINITY;
    chk(cudaMemcpy(s->lo64, inf.data(), sizeof(double) * s->tot_n, cudaMemcpyHostToDevice));
    chk(launch_convert(s->lo64, s->tot_n, precision, s->lo_T, 0));
    chk(cudaDeviceSynchronize());
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("device initialisation failed: ") + cudaGetErrorString(e);
    pimpc_destroy(s);
    return PIMPC_ECUDA;
  }
  Layout &L = s->L;
  L.batch = batch; L.lti = lti; L.nx = d_nx; L.nu = d_nu; L.N = d_N;
  L.off_nx = d_off[0]; L.off_nu = d_off[1]; L.off_n = d_off[2];
  L.Nnx = d_off[3]; L.Nnu = d_off[4]; L.Nn = d_off[5];
  L.offA = d_off[6]; L.offB = d_off[7]; L.offe = d_off[8];
  L.stage0 = d_off[9];
  std::string why;
  const int rc = apply_schedule(s, Schedule{}, why);
  if (rc != PIMPC_OK) {
    g_create_error = why;
    pimpc_destroy(s);
    return rc;
  }
  *out = s;
  return PIMPC_OK;
}

int pimpc_set_options(pimpc_solver *s, double rho, double eps, int max_iters, int accel,
                      double eta) {
  if (!s) return PIMPC_EINVAL;
  if (!(rho > 0.0) || !std::isfinite(rho)) return fail(s, PIMPC_EINVAL, "rho must be > 0");
  if (std::isnan(eps)) return fail(s, PIMPC_EINVAL, "eps is NaN");
  if (max_iters < 0) return fail(s, PIMPC_EINVAL, "max_iters < 0");
  if (accel != 0 && accel != 1) return fail(s, PIMPC_EINVAL, "accel must be 0 or 1");
  if (!(eta >= 0.0) || !std::isfinite(eta)) return fail(s, PIMPC_EINVAL, "eta must be >= 0");
  if (s->mask && s->mask_len > max_iters) return fail(s, PIMPC_EINVAL, "restart mask longer than max_iters");
  if (rho != s->rho) {
    s->stale = true;
    ++s->fgen;
  }
  s->rho = rho; s->eps = eps; s->max_iters = max_iters; s->accel = accel; s->eta = eta;
  graph_invalidate(s);
  if (const int rc = ensure_coef_table(s)) return rc;
  return PIMPC_OK;
}

int pimpc_set_weights(pimpc_solver *s, const double *q, const double *r, const double *rdu,
                      int mem, void *stream) {
  if (!s || !q || !r) return fail(s, PIMPC_EINVAL, "q and r are required");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  if (mem == PIMPC_HOST) {
    for (int64_t i = 0; i < s->tot_nx; ++i)
      if (!(q[i] >= 0.0) || !std::isfinite(q[i])) return fail(s, PIMPC_EINVAL, "q must be finite and >= 0");
    for (int64_t i = 0; i < s->tot_nu; ++i) {
      if (!(r[i] >= 0.0) || !std::isfinite(r[i])) return fail(s, PIMPC_EINVAL, "r must be finite and >= 0");
      if (rdu && (!(rdu[i] >= 0.0) || !std::isfinite(rdu[i])))
        return fail(s, PIMPC_EINVAL, "rdu must be finite and >= 0");
    }
  }
  const double *dq, *dr, *drdu;
  PIMPC_CHECK(s, dev_in(s, q, s->tot_nx, mem, 0, st, &dq), "copy q");
  PIMPC_CHECK(s, dev_in(s, r, s->tot_nu, mem, s->tot_nx, st, &dr), "copy r");
  PIMPC_CHECK(s, dev_in(s, rdu, s->tot_nu, mem, s->tot_nx + s->tot_nu, st, &drdu), "copy rdu");
  PIMPC_CHECK(s, launch_gather_n64(s->L, dq, dr, s->tot_n, s->qd64, st), "weights");
  PIMPC_CHECK(s, launch_gather_n(s->L, dq, dr, s->tot_n, s->prec, s->qd_T, st), "weights");
  PIMPC_CHECK(s, launch_gather_n64(s->L, nullptr, drdu, s->tot_n, s->rdu64, st), "weights");
  s->have_rdu = rdu != nullptr;
  s->stale = true;
  ++s->fgen;
  if (mem == PIMPC_HOST) PIMPC_CHECK(s, cudaStreamSynchronize(st), "set_weights");
  return PIMPC_OK;
}

int pimpc_set_bounds(pimpc_solver *s, const double *xmin, const double *xmax, const double *umin,
                     const double *umax, int mem, void *stream) {
  if (!s || !xmin || !xmax || !umin || !umax) return fail(s, PIMPC_EINVAL, "all four bounds are required");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  if (mem == PIMPC_HOST) {
    if (!finite_or_inf_ok(xmin, s->tot_nx) || !finite_or_inf_ok(xmax, s->tot_nx) ||
        !finite_or_inf_ok(umin, s->tot_nu) || !finite_or_inf_ok(umax, s->tot_nu))
      return fail(s, PIMPC_EINVAL, "NaN bound");
    for (int64_t i = 0; i < s->tot_nx; ++i)
      if (xmin[i] > xmax[i]) return fail(s, PIMPC_EINVAL, "xmin > xmax");
    for (int64_t i = 0; i < s->tot_nu; ++i)
      if (umin[i] > umax[i]) return fail(s, PIMPC_EINVAL, "umin > umax");
  }
  const double *a, *b, *c, *d;
  int64_t o = 0;
  PIMPC_CHECK(s, dev_in(s, xmin, s->tot_nx, mem, o, st, &a), "copy bounds"); o += s->tot_nx;
  PIMPC_CHECK(s, dev_in(s, xmax, s->tot_nx, mem, o, st, &b), "copy bounds"); o += s->tot_nx;
  PIMPC_CHECK(s, dev_in(s, umin, s->tot_nu, mem, o, st, &c), "copy bounds"); o += s->tot_nu;
  PIMPC_CHECK(s, dev_in(s, umax, s->tot_nu, mem, o, st, &d), "copy bounds");
  PIMPC_CHECK(s, launch_gather_n(s->L, a, c, s->tot_n, s->prec, s->lo_T, st), "bounds");
  PIMPC_CHECK(s, launch_gather_n(s->L, b, d, s->tot_n, s->prec, s->hi_T, st), "bounds");
  PIMPC_CHECK(s, launch_gather_n64(s->L, a, c, s->tot_n, s->lo64, st), "bounds");
  PIMPC_CHECK(s, launch_gather_n64(s->L, b, d, s->tot_n, s->hi64, st), "bounds");
  if (mem == PIMPC_HOST) PIMPC_CHECK(s, cudaStreamSynchronize(st), "set_bounds");
  return PIMPC_OK;
}

int pimpc_set_dynamics(pimpc_solver *s, const double *A, const double *B, const double *e,
                       int mem, void *stream) {
  if (!s || !A || !B) return fail(s, PIMPC_EINVAL, "A and B are required");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  const cudaMemcpyKind kind = mem == PIMPC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  PIMPC_CHECK(s, cudaMemcpyAsync(s->A64, A, sizeof(double) * s->tot_A, kind, st), "copy A");
  PIMPC_CHECK(s, cudaMemcpyAsync(s->B64, B, sizeof(double) * s->tot_B, kind, st), "copy B");
  if (e) PIMPC_CHECK(s, cudaMemcpyAsync(s->e64, e, sizeof(double) * s->tot_e, kind, st), "copy e");
  else PIMPC_CHECK(s, cudaMemsetAsync(s->e64, 0, sizeof(double) * s->tot_e, st), "zero e");
  s->stale = true;
  ++s->fgen;
  if (mem == PIMPC_HOST) PIMPC_CHECK(s, cudaStreamSynchronize(st), "set_dynamics");
  return PIMPC_OK;
}

int pimpc_linearise(pimpc_solver *s, int model, const double *params, double dt,
                    const double *xbar, const double *ubar, int mem, void *stream) {
  if (!s || !params || !xbar || !ubar) return fail(s, PIMPC_EINVAL, "params, xbar and ubar are required");
  int mnx, mnu;
  if (model_dims(model, &mnx, &mnu)) return fail(s, PIMPC_EINVAL, "unknown model");
  for (int j = 0; j < s->batch; ++j)
    if (s->nx[j] != mnx || s->nu[j] != mnu) return fail(s, PIMPC_EINVAL, "instance sizes do not match the model");
  if (!(dt > 0.0)) return fail(s, PIMPC_EINVAL, "dt must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  const int64_t npts = s->lti ? s->batch : s->nblocks;
  const int64_t nxp = s->lti ? s->tot_nx : s->tot_Nnx, nup = s->lti ? s->tot_nu : s->tot_Nnu;
  const double *dx, *du, *dp;
  PIMPC_CHECK(s, dev_in(s, xbar, nxp, mem, 0, st, &dx), "copy xbar");
  PIMPC_CHECK(s, dev_in(s, ubar, nup, mem, nxp, st, &du), "copy ubar");
  PIMPC_CHECK(s, dev_in(s, params, (int64_t)s->batch * model_nparams(model), mem, nxp + nup, st, &dp), "copy params");
  PIMPC_CHECK(s, launch_linearise(s->L, model, dp, dt, dx, du, s->A64, s->B64, s->e64, npts,
                                  s->lti ? nullptr : s->binst, s->lti ? nullptr : s->d_bbase, st),
              "linearise");
  s->stale = true;
  ++s->fgen;
  if (mem == PIMPC_HOST) PIMPC_CHECK(s, cudaStreamSynchronize(st), "linearise");
  return PIMPC_OK;
}

int pimpc_get_dynamics(pimpc_solver *s, double *A, double *B, double *e, int mem, void *stream) {
  if (!s) return PIMPC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  const cudaMemcpyKind kind = mem == PIMPC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (A) PIMPC_CHECK(s, cudaMemcpyAsync(A, s->A64, sizeof(double) * s->tot_A, kind, st), "copy A");
  if (B) PIMPC_CHECK(s, cudaMemcpyAsync(B, s->B64, sizeof(double) * s->tot_B, kind, st), "copy B");
  if (e) PIMPC_CHECK(s, cudaMemcpyAsync(e, s->e64, sizeof(double) * s->tot_e, kind, st), "copy e");
  if (mem == PIMPC_HOST) PIMPC_CHECK(s, cudaStreamSynchronize(st), "get_dynamics");
  return PIMPC_OK;
}

int pimpc_factorise(pimpc_solver *s, void *stream) {
  if (!s) return PIMPC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  PIMPC_CHECK(s, launch_factorise(s->L, s->A64, s->B64, s->e64, s->qd64,
                                  s->have_rdu ? s->rdu64 : nullptr, s->rho, s->binst, s->d_bbase,
                                  s->nblocks, s->max_nx, s->max_n, s->prec, s->blk_T, s->ferr, st),
              "factorise");
  s->stale = false;
  return PIMPC_OK;
}

int pimpc_set_graph(pimpc_solver *s, int enable) {
  if (!s) return PIMPC_EINVAL;
  if (enable != 0 && enable != 1) return fail(s, PIMPC_EINVAL, "enable must be 0 or 1");
  cudaSetDevice(s->device);
  graph_invalidate(s);
  s->graph_on = enable;
  s->graph_failed = 0;
  s->graph_err.clear();
  return PIMPC_OK;
}

int pimpc_get_graph_stats(pimpc_solver *s, int *enabled, long long *captures, long long *replays,
                          const char **refused) {
  if (!s) return PIMPC_EINVAL;
  if (enabled) *enabled = s->graph_on && !s->graph_failed;
  if (captures) *captures = s->graph_captures;
  if (replays) *replays = s->graph_replays;
  if (refused) *refused = s->graph_failed ? s->graph_err.c_str() : nullptr;
  return PIMPC_OK;
}

int pimpc_set_polish(pimpc_solver *s, int polish_iters, double polish_eps) {
  if (!s) return PIMPC_EINVAL;
  if (polish_iters < 0) return fail(s, PIMPC_EINVAL, "polish_iters < 0");
  if (std::isnan(polish_eps)) return fail(s, PIMPC_EINVAL, "polish_eps is NaN");
  s->polish_iters = polish_iters;
  s->polish_eps = polish_eps;
  graph_invalidate(s);
  return PIMPC_OK;
}

int pimpc_solve(pimpc_solver *s, const double *x0, const double *u_prev, const double *ref,
                int ref_per_stage, int warm_start, double *u_out, double *x_out, int *iters,
                double *c, int *status, int mem, void *stream) {
  if (!s || !x0) return fail(s, PIMPC_EINVAL, "x0 is required");
  if (warm_start < 0 || warm_start > 2) return fail(s, PIMPC_EINVAL, "warm_start must be 0, 1 or 2");
  if (ref_per_stage != 0 && ref_per_stage != 1) return fail(s, PIMPC_EINVAL, "ref_per_stage must be 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  const double *dx0, *dup, *dref;
  const int64_t nref = ref_per_stage ? s->tot_Nn : s->tot_n;
  PIMPC_CHECK(s, dev_in(s, x0, s->tot_nx, mem, 0, st, &dx0), "copy x0");
  PIMPC_CHECK(s, dev_in(s, u_prev, s->tot_nu, mem, s->tot_nx, st, &dup), "copy u_prev");
  PIMPC_CHECK(s, dev_in(s, ref, nref, mem, s->tot_nx + s->tot_nu, st, &dref), "copy ref");
  const bool dev = mem == PIMPC_DEVICE;
  double *u_dev = u_out ? (dev ? u_out : s->out_u) : nullptr;
  double *x_dev = x_out ? (dev ? x_out : s->out_x) : nullptr;
  const bool polish = s->polish_iters > 0 && s->prec == PIMPC_F32;
  if (dev && s->graph_on && !s->graph_failed) {
    const int rc = graph_solve(s, dx0, dup, dref, ref_per_stage, warm_start, u_dev, x_dev, iters,
                               c, status, polish, st);
    if (rc != PIMPC_OK || !s->graph_failed) return rc;
    // the capture was refused: this call and the later ones run the launches directly
  }
  int rc = run_solve(s, dx0, dup, dref, ref_per_stage, warm_start, polish ? nullptr : u_dev,
                     polish ? nullptr : x_dev, st);
  if (rc != PIMPC_OK) return rc;
  if (polish) {
    rc = prepare_polish(s, st);
    if (rc == PIMPC_OK) rc = polish_launch(s, dx0, dup, dref, ref_per_stage, u_dev, x_dev, st);
    if (rc != PIMPC_OK) return rc;
  }
  s->last_polished = polish;
  if (dev) {
    if (iters || c || status)
      PIMPC_CHECK(s, launch_unpack_state(s->st, s->batch, iters, c, status, nullptr, st), "state");
    return PIMPC_OK;
  }
  if (u_out) PIMPC_CHECK(s, cudaMemcpyAsync(u_out, s->out_u, sizeof(double) * s->tot_Nnu, cudaMemcpyDeviceToHost, st), "copy u");
  if (x_out) PIMPC_CHECK(s, cudaMemcpyAsync(x_out, s->out_x, sizeof(double) * s->tot_Nnx, cudaMemcpyDeviceToHost, st), "copy x");
  if (iters || c || status) {
    std::vector<InstState> hs(s->batch);
    PIMPC_CHECK(s, cudaMemcpyAsync(hs.data(), s->st, sizeof(InstState) * s->batch, cudaMemcpyDeviceToHost, st), "copy state");
    PIMPC_CHECK(s, cudaStreamSynchronize(st), "solve");
    for (int j = 0; j < s->batch; ++j) {
      if (iters) iters[j] = hs[j].iters;
      if (c) c[j] = hs[j].c;
      if (status) status[j] = hs[j].status;
    }
  } else {
    PIMPC_CHECK(s, cudaStreamSynchronize(st), "solve");
  }
  return PIMPC_OK;
}

int pimpc_get_iterates(pimpc_solver *s, double *z, double *v, double *theta, double *beta,
                       double *lambda, int mem, void *stream) {
  if (!s) return PIMPC_EINVAL;
  if (!s->solved) return fail(s, PIMPC_ESTATE, "no solve has run");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  double *outs[5] = {z, v, theta, beta, lambda};
  if (mem == PIMPC_DEVICE) {
    PIMPC_CHECK(s, launch_export_iterates(s->L, s->it, s->base, s->prec, z, v, theta, beta, lambda, st),
                "export");
    return PIMPC_OK;
  }
  for (int b = 0; b < 5; ++b) {
    if (!outs[b]) continue;
    double *tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    tmp[b] = s->stage64;
    PIMPC_CHECK(s, launch_export_iterates(s->L, s->it, s->base, s->prec, tmp[0], tmp[1], tmp[2],
                                          tmp[3], tmp[4], st), "export");
    PIMPC_CHECK(s, cudaMemcpyAsync(outs[b], s->stage64, sizeof(double) * s->tot_Nn, cudaMemcpyDeviceToHost, st), "copy iterates");
    PIMPC_CHECK(s, cudaStreamSynchronize(st), "get_iterates");
  }
  return PIMPC_OK;
}

int pimpc_get_stats(pimpc_solver *s, int *iters, double *c, int *status, int *momentum_iters,
                    int mem, void *stream) {
  if (!s) return PIMPC_EINVAL;
  if (!s->solved) return fail(s, PIMPC_ESTATE, "no solve has run");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  if (mem == PIMPC_DEVICE) {
    PIMPC_CHECK(s, launch_unpack_state(s->st, s->batch, iters, c, status, momentum_iters, st), "stats");
    return PIMPC_OK;
  }
  std::vector<InstState> hs(s->batch);
  PIMPC_CHECK(s, cudaMemcpyAsync(hs.data(), s->st, sizeof(InstState) * s->batch, cudaMemcpyDeviceToHost, st), "copy stats");
  PIMPC_CHECK(s, cudaStreamSynchronize(st), "get_stats");
  for (int j = 0; j < s->batch; ++j) {
    if (iters) iters[j] = hs[j].iters;
    if (c) c[j] = hs[j].c;
    if (status) status[j] = hs[j].status;
    if (momentum_iters) momentum_iters[j] = hs[j].momentum;
  }
  return PIMPC_OK;
}

int pimpc_set_restart_mask(pimpc_solver *s, const unsigned char *mask, int len, int mem,
                           void *stream) {
  if (!s) return PIMPC_EINVAL;
  cudaSetDevice(s->device);
  cudaStream_t st = (cudaStream_t)stream;
  graph_invalidate(s);
  if (!mask) { s->mask_len = 0; s->mask = nullptr; return PIMPC_OK; }
  if (len < 0 || len > s->max_iters) return fail(s, PIMPC_EINVAL, "mask length must be in [0, max_iters]");
  // Testing aid: the mask buffer is (re)allocated here, sized for this mask.
  const size_t bytes = (size_t)s->batch * (size_t)std::max(len, 1);
  if (s->mask_alloc) { cudaFree(s->mask_alloc); s->mask_alloc = nullptr; }
  unsigned char *buf = nullptr;
  PIMPC_CHECK(s, cudaMalloc((void **)&buf, bytes), "mask allocation");
  s->mask_alloc = buf;
  const cudaMemcpyKind kind = mem == PIMPC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  PIMPC_CHECK(s, cudaMemcpyAsync(buf, mask, (size_t)s->batch * len, kind, st), "copy mask");
  if (mem == PIMPC_HOST) PIMPC_CHECK(s, cudaStreamSynchronize(st), "mask");
  s->mask = buf;
  s->mask_len = len;
  return PIMPC_OK;
}

}  // extern "C"

namespace pimpc {
// Input sets from host arrays (validated): kind [batch], r [batch], a [sum nu] (may be null).
int store_input_sets(pimpc_solver *s, const int *kind, const double *r, const double *a,
                     cudaStream_t st) {
  bool any = false;
  for (int j = 0; j < s->batch; ++j) {
    const int k = kind[j];
    if (k < 0 || k > 4) return fail(s, PIMPC_EINVAL, "input set kind must be 0..4");
    if (k == 0) continue;
    any = true;
    if (!std::isfinite(r[j]) || ((k == 1 || k == 2) && r[j] < 0.0))
      return fail(s, PIMPC_EINVAL, "input set: r must be finite (and >= 0 for a ball)");
    if (k == 3) {
      if (!a) return fail(s, PIMPC_EINVAL, "halfspace input set needs its normal a");
      double nn = 0.0;
      for (int i = 0; i < s->nu[j]; ++i) {
        const double v = a[s->off_nu[j] + i];
        if (!std::isfinite(v)) return fail(s, PIMPC_EINVAL, "input set: non-finite normal");
        nn += v * v;
      }
      if (!(nn > 0.0)) return fail(s, PIMPC_EINVAL, "input set: zero halfspace normal");
    }
  }
  if (any && s->sched.family != 0 && s->sched.family != 5)
    return fail(s, PIMPC_EINVAL, "non-box input sets need schedule family 0 or 5");
  const size_t ts = s->prec == PIMPC_F32 ? 4 : 8;
  if (!s->uset_kind_d) {
    cudaError_t e = cudaMalloc((void **)&s->uset_kind_d, sizeof(int) * s->batch);
    if (e == cudaSuccess) e = cudaMalloc(&s->uset_r_T, ts * s->batch);
    if (e == cudaSuccess) e = cudaMalloc(&s->uset_a_T, ts * s->tot_n);
    if (e != cudaSuccess) return fail(s, PIMPC_ENOMEM, "input set arrays");
  }
  s->uset_kind_h.assign(kind, kind + s->batch);
  s->uset_r_h.assign(r, r + s->batch);
  if (a) s->uset_a_h.assign(a, a + s->tot_nu);
  else s->uset_a_h.assign(s->tot_nu, 0.0);
  PIMPC_CHECK(s, cudaMemcpyAsync(s->uset_kind_d, s->uset_kind_h.data(), sizeof(int) * s->batch,
                                 cudaMemcpyHostToDevice, st), "input set kinds");
  double *tmp = nullptr;  // FP64 staging for the conversion, freed before returning
  PIMPC_CHECK(s, cudaMalloc((void **)&tmp, sizeof(double) * (s->batch + s->tot_nu)),
              "input set staging");
  PIMPC_CHECK(s, cudaMemcpyAsync(tmp, s->uset_r_h.data(), sizeof(double) * s->batch,
                                 cudaMemcpyHostToDevice, st), "input set radii");
  PIMPC_CHECK(s, cudaMemcpyAsync(tmp + s->batch, s->uset_a_h.data(), sizeof(double) * s->tot_nu,
                                 cudaMemcpyHostToDevice, st), "input set normals");
  PIMPC_CHECK(s, launch_convert(tmp, s->batch, s->prec, s->uset_r_T, st), "input set radii");
  PIMPC_CHECK(s, launch_gather_n(s->L, nullptr, tmp + s->batch, s->tot_n, s->prec, s->uset_a_T, st),
              "input set normals");
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(tmp);
  PIMPC_CHECK(s, e2, "input sets");
  s->any_uset = any;
  graph_invalidate(s);
  return PIMPC_OK;
}
}  // namespace pimpc

extern "C" {

int pimpc_set_input_set(pimpc_solver *s, const int *kind, const double *r, const double *a,
                        int mem, void *stream) {
  if (!s || !kind || !r) return fail(s, PIMPC_EINVAL, "kind and r are required");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  if (mem == PIMPC_HOST) return store_input_sets(s, kind, r, a, st);
  // device arrays: validated on host copies (a setup call, not on the solve path)
  std::vector<int> kh(s->batch);
  std::vector<double> rh(s->batch), ah(a ? s->tot_nu : 0);
  PIMPC_CHECK(s, cudaMemcpyAsync(kh.data(), kind, sizeof(int) * s->batch, cudaMemcpyDeviceToHost, st), "copy kinds");
  PIMPC_CHECK(s, cudaMemcpyAsync(rh.data(), r, sizeof(double) * s->batch, cudaMemcpyDeviceToHost, st), "copy r");
  if (a) PIMPC_CHECK(s, cudaMemcpyAsync(ah.data(), a, sizeof(double) * s->tot_nu, cudaMemcpyDeviceToHost, st), "copy a");
  PIMPC_CHECK(s, cudaStreamSynchronize(st), "input sets");
  return store_input_sets(s, kh.data(), rh.data(), a ? ah.data() : nullptr, st);
}

int pimpc_set_stall(pimpc_solver *s, int window, double factor, double below, double rel) {
  if (!s) return PIMPC_EINVAL;
  if (window < 0) return fail(s, PIMPC_EINVAL, "window must be >= 0");
  if (!(factor > 0.0 && factor <= 1.0)) return fail(s, PIMPC_EINVAL, "factor must be in (0, 1]");
  if (!(below >= 0.0)) return fail(s, PIMPC_EINVAL, "below must be >= 0");
  if (!(rel >= 0.0) || !std::isfinite(rel)) return fail(s, PIMPC_EINVAL, "rel must be >= 0");
  graph_invalidate(s);
  s->stall_win = window;
  s->stall_fac = factor;
  s->stall_below = below;
  s->stall_rel = rel;
  return PIMPC_OK;
}

int pimpc_set_wait_limit(pimpc_solver *s, int polls) {
  if (!s) return PIMPC_EINVAL;
  if (polls < 0) return fail(s, PIMPC_EINVAL, "polls must be >= 0");
  graph_invalidate(s);
  s->bar_limit = polls;
  return PIMPC_OK;
}

int pimpc_plant_step(pimpc_solver *s, int model, const double *params, double dt,
                     const double *x, const double *u, double *x_next, int mem, void *stream) {
  if (!s || !params || !x || !u || !x_next) return fail(s, PIMPC_EINVAL, "missing argument");
  int mnx, mnu;
  if (model_dims(model, &mnx, &mnu)) return fail(s, PIMPC_EINVAL, "unknown model");
  for (int j = 0; j < s->batch; ++j)
    if (s->nx[j] != mnx || s->nu[j] != mnu) return fail(s, PIMPC_EINVAL, "instance sizes do not match the model");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  const double *dx, *du, *dp;
  int64_t o = 0;
  PIMPC_CHECK(s, dev_in(s, x, s->tot_nx, mem, o, st, &dx), "copy x"); o += s->tot_nx;
  PIMPC_CHECK(s, dev_in(s, u, s->tot_nu, mem, o, st, &du), "copy u"); o += s->tot_nu;
  PIMPC_CHECK(s, dev_in(s, params, (int64_t)s->batch * model_nparams(model), mem, o, st, &dp), "copy params");
  o += (int64_t)s->batch * model_nparams(model);
  double *dxn = mem == PIMPC_DEVICE ? x_next : s->stage64 + o;
  PIMPC_CHECK(s, launch_plant_step(s->L, model, dp, dt, dx, du, dxn, st), "plant step");
  if (mem == PIMPC_HOST) {
    PIMPC_CHECK(s, cudaMemcpyAsync(x_next, dxn, sizeof(double) * s->tot_nx, cudaMemcpyDeviceToHost, st), "copy x_next");
    PIMPC_CHECK(s, cudaStreamSynchronize(st), "plant step");
  }
  return PIMPC_OK;
}

}  // extern "C"

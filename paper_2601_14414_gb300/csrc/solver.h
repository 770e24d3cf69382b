// solver.h -- the solver object behind the opaque pimpc_solver handle (internal to the library).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "launch.h"

struct pimpc_solver {
  int device = 0, batch = 0, lti = 0, prec = 0, tiled = 1;
  std::vector<int> nx, nu, N, W, tw;
  pimpc::Schedule sched{};
  int res_plan[6] = {0, 0, 0, 0, 0, 0};   // resident schedule: cluster size and smem regions
  int gemm_plan[5] = {0, 0, 0, 0, 0};     // contraction schedule: stages per item, padding
  double *coef_tab = nullptr;             // momentum factors by streak length (resident)
  int coef_len = 0;
  std::vector<void *> lay_allocs;   // buffers whose size depends on the schedule
  std::vector<int64_t> off_nx, off_nu, off_n, Nnx, Nnu, Nn, Ni, offA, offB, offe, blk, stage0, bbase;
  int64_t tot_nx = 0, tot_nu = 0, tot_n = 0, tot_Nnx = 0, tot_Nnu = 0, tot_Nn = 0, tot_Ni = 0;
  int64_t tot_A = 0, tot_B = 0, tot_e = 0, tot_blk = 0, nblocks = 0, stage_words = 0;
  int max_nx = 0, max_n = 0;
  pimpc::Layout L{};
  std::vector<void *> allocs;
  // device buffers
  double *A64 = nullptr, *B64 = nullptr, *e64 = nullptr;
  double *qd64 = nullptr, *rdu64 = nullptr, *stage64 = nullptr;
  double *out_u = nullptr, *out_x = nullptr;
  void *blk_T = nullptr, *qd_T = nullptr, *ref_T = nullptr;
  void *it[3] = {nullptr, nullptr, nullptr};
  void *lo_T = nullptr, *hi_T = nullptr, *xb0_T = nullptr;
  int *base = nullptr, *old_base = nullptr, *binst = nullptr, *ferr = nullptr;  // ferr: [batch]
  double *alpha = nullptr, *cprev = nullptr, *coef = nullptr, *cacc = nullptr;
  int *ndone = nullptr, *stop = nullptr;
  int *item_inst = nullptr, *item_a = nullptr, *item_b = nullptr, *nitems_inst = nullptr;
  int *list0 = nullptr, *list1 = nullptr;
  int *item_first = nullptr;  // [2 batch] first coarse / fine item of each instance
  double *cpart = nullptr;    // [items] per-item share of c of the current iteration
  int *list_init = nullptr;   // [coarse items] starting order of the active list
  int *ccount = nullptr;      // [grid] per-CTA counts of the order-keeping compaction
  int *pos_of = nullptr;      // [items] position of each item in the active list
  pimpc::Ctl *ctl = nullptr;
  int64_t *d_bbase = nullptr;
  pimpc::InstState *st = nullptr;
  unsigned char *mask = nullptr, *mask_alloc = nullptr;
  int mask_len = 0;
  int bar_limit = 0;  // grid-barrier polls before a launch gives up (0: the built-in limit)
  int stall_win = 0;  // stall stop: window (0: off) and factor, per-instance best c / iteration
  double stall_fac = 0.5, stall_below = 1e-9, stall_rel = 0.0;
  int *itfirst = nullptr;
  float *tc_mat = nullptr;       // tensor-core schedule: per-instance matrix blocks
  int64_t *tc_off = nullptr;     // [batch] word offsets of those blocks
  int tb_T = 8;  // temporal blocking: iterations per block
  double *cbest = nullptr;
  int *itbest = nullptr;
  // input sets (pimpc_set_input_set): device kind [batch], r [batch] and normal [sum n] in the
  // iteration precision (x slots 0), allocated by the first call; host copies for the polish
  bool any_uset = false;
  int *uset_kind_d = nullptr;
  void *uset_r_T = nullptr, *uset_a_T = nullptr;
  std::vector<int> uset_kind_h;
  std::vector<double> uset_r_h, uset_a_h;  // r [batch], a [sum nu]
  int nitems = 0;
  // options and state
  double rho = 1.0, eps = 1e-6, eta = 0.999;
  int max_iters = 1000, accel = 1;
  bool stale = true, have_rdu = false, solved = false;
  int last_ref_per_stage = 0, last_ref_given = 0, last_warm = 0, last_accel = 0, last_iters_fixed = 0;
  double last_eps = 0.0;
  size_t smem_admm = 0;
  int grid_admm = 0;
  pimpc::AdmmLaunch plan{};
  std::string err;
  // FP64 polish: FP64 bounds, options, and the FP64 solver that runs the polish iterations
  // (created by the first polished solve; it reads this solver's FP64 dynamics and weights)
  double *lo64 = nullptr, *hi64 = nullptr;
  int polish_iters = 0;
  double polish_eps = 0.0;
  pimpc_solver *shadow = nullptr;
  long fgen = 0, shadow_fgen = -1;   // generation of the factorisation inputs
  bool last_polished = false;
  // CUDA graphs of device-memory solves: one per argument set, replayed on later calls; every
  // call that changes launch parameters drops them
  struct GraphEntry {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec;
    int warm, ref_per_stage, ref_given, polished;
  };
  int graph_on = 0, graph_failed = 0;
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  long graph_captures = 0, graph_replays = 0;
  std::string graph_err;
  // adjoint workspace (allocated by the first pimpc_backward)
  void *adj_ws = nullptr;
  size_t adj_ws_bytes = 0;
};

namespace pimpc {
int fail(pimpc_solver *s, int code, const std::string &msg);
int ensure_coef_table(pimpc_solver *s);
void graph_invalidate(pimpc_solver *s);
int apply_schedule(pimpc_solver *s, const Schedule &sc, std::string &why);
int cuda_fail(pimpc_solver *s, cudaError_t e, const char *what);
size_t tsize(int prec);
cudaError_t dev_in(pimpc_solver *s, const double *p, int64_t count, int mem, int64_t at,
                   cudaStream_t st, const double **out);
}  // namespace pimpc

#define PIMPC_CHECK(s, expr, what)                                       \
  do {                                                                   \
    cudaError_t _e = (expr);                                             \
    if (_e != cudaSuccess) return pimpc::cuda_fail((s), _e, (what));     \
  } while (0)

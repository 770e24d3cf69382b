// launch.h -- host-side launchers of the library's kernels (internal to the library).
#pragma once
#include "pimpc_internal.cuh"

namespace pimpc {

int factorise_smem_words(int max_nx, int max_n);
cudaError_t launch_factorise(const Layout &L, const double *A, const double *B, const double *e,
                             const double *qd, const double *rdu, double rho, const int *binst,
                             const int64_t *bbase, int64_t nblocks, int max_nx, int max_n,
                             int precision, void *blk, int *err, cudaStream_t stream);

struct AdmmLaunch {
  Layout L;
  const void *blk;
  void *it[3];
  const void *qd, *ref;
  int ref_per_stage;
  const void *lo, *hi, *xb0;
  double rho, eps, eta;
  int max_iters, accel;
  const unsigned char *mask;
  int mask_len;
  // work items
  const int *item_inst, *item_a, *item_b, *nitems_inst;
  int nitems;
  // per instance the first coarse and the first fine item ([2 batch]; null: c accumulates by
  // atomics in finish_item), and the per-item shares of c of the current iteration
  const int *item_first;
  double *cpart;
  // the active list's starting order (longest items first) and the per-CTA counts of the
  // order-keeping compaction (null: item order, and a compaction that keeps no order)
  const int *list_init;
  int *ccount;
  int *pos_of;      // [items] position of each item in the active list (null: stopped
                    // instances leave the list at the next iteration's compaction)
  // fine items (one sub-chunk each) after the nitems coarse ones: nfine of them from index
  // nfine_base; nitems_inst holds the coarse then the fine per-instance counts (0: none)
  int nfine_base, nfine, fine_switch;
  int *list0, *list1;
  Ctl *ctl;
  // per-instance state
  int *base, *old_base;
  InstState *st;
  double *alpha, *cprev, *coef, *cacc;
  int *ndone, *stop;
  double *u_out, *x_out;
  const double *coef_tab;
  const int *grp;   // blocked kernel: lane groups per sub-chunk of each instance
  int warm;
  const int *ferr;  // [batch] nonzero: the instance's factorisation met a non-positive pivot
  // input sets (null: the box for every instance): kind [batch], r [batch], a [sum n] (type T)
  const int *uset_kind;
  const void *uset_r, *uset_a;
  // stop at the arithmetic's floor: once c <= stall_below (first at iteration i0), no c below
  // stall_fac x the best c for max(stall_win, stall_rel x i0) iterations
  int stall_win;    // 0: off (Algorithm 1's stop test only)
  double stall_fac, stall_below, stall_rel;
  double *cbest;    // [batch] best c so far, and the iteration that set it
  int *itbest;
  int *itfirst;     // [batch] i0 (-1: c not yet below stall_below)
  int bar_limit;    // grid-barrier polls before giving up (0: the default limit)
  // launch shape and shared-memory plan (elements of the iteration type)
  int grid, threads;
  int capB, capI, haloB, haloI, S_max, nv_max, nbuf;
};

__global__ void set_control_kernel(Ctl *c, int nitems, int batch, int bar_limit);
int admm_threads(int precision);
int admm_iter_stride(int n, int precision);
int admm_group_size(int n);
size_t admm_smem_bytes(const AdmmLaunch &s, int precision);
cudaError_t admm_configure(int precision, size_t smem, int *blocks_per_sm);
cudaError_t launch_admm(const AdmmLaunch &a, int precision, cudaStream_t stream);

// One thread per stage on halo tiles (stage-varying FP32 instances).
int tile_threads();
int tile_warps();
cudaError_t tile_configure(size_t smem, int *blocks_per_sm);
cudaError_t launch_tile(const AdmmLaunch &a, cudaStream_t stream);

// Every instance resident on chip: one CTA or a cluster of C CTAs per instance.
int res_threads(int precision);
cudaError_t launch_coef_table(double *tab, int len, cudaStream_t stream);
size_t res_plan(int batch, const int *nx, const int *nu, const int *N, const int *W, int lti,
                int precision, int threads, int C, int *plan);
cudaError_t launch_resident(const AdmmLaunch &s, int precision, const int *plan, size_t smem,
                            cudaStream_t stream);

// Stage-invariant instances as dense contractions (register-tiled products over stage blocks).
int gemm_threads();
int gemm_plan(int max_n, int max_nx, int max_nu, int precision, size_t budget, int *plan);
cudaError_t gemm_configure(int precision, size_t smem, int *blocks_per_sm);
cudaError_t launch_gemm(const AdmmLaunch &s, int precision, const int *plan, cudaStream_t stream);

// Lane groups owning 4-column blocks on blocked stage blocks (tiled == 3).
int blk_threads();
// Shared-memory elements of a sub-chunk of S lane groups (S - 1 stages and the next stage).
int64_t blk_region_words(int nx, int nu, int lti, int precision, int S);
cudaError_t blk_configure(int precision, size_t smem, int *blocks_per_sm);
cudaError_t launch_blk(const AdmmLaunch &a, int precision, size_t smem, cudaStream_t stream);

// Stage-invariant FP32 instances with the stage products on the tensor cores (tiled == 4).
int tc_threads();
bool tc_fits(int nx, int nu);
int64_t tc_block_words(int nx, int nu);
size_t tc_smem_bytes(int nx, int nu);
cudaError_t tc_configure(size_t smem, int *blocks_per_sm);
cudaError_t launch_tc(const AdmmLaunch &s, const float *tcm, const int64_t *tc_off, size_t smem,
                      cudaStream_t stream);

// Temporal blocking of the plain iteration: windows of stages iterated T times in shared memory.
int tb_threads();
int64_t tb_window_words(int nx, int nu, int W, int lti, int precision, int S);
size_t tb_static_smem(int precision);  // the kernel's static shared memory (bytes)
cudaError_t tb_configure(int precision, size_t smem, int *blocks_per_sm);
cudaError_t launch_tb(const AdmmLaunch &s, int precision, int T, size_t smem, cudaStream_t stream);

// Schedule of the batched solve: which kernel family and how its work is cut.
struct Schedule {
  int family = -1;       // 0: lane groups on plain stage blocks; 2: one thread per stage on halo
                         // tiles (stage-varying FP32 only); 3: every instance resident in the
                         // shared memory of one CTA or a cluster (item_scale = CTAs per
                         // instance, 0: the fewest that fit); 4: stage-invariant instances as
                         // dense contractions over blocks of stages; 5: lane groups owning
                         // 4-column blocks on blocked stage blocks; 6: stage-invariant FP32
                         // instances with the stage products on the tensor cores; 7: temporal
                         // blocking of the plain iteration (item_scale = T); -1: the default
  int ctas_per_sm = 0;   // halo tiles and blocked lane groups: CTAs per SM the shared-memory
                         // budget is sized for (0: 2 for halo tiles, 3 for blocked lane groups)
  int item_scale = 0;    // lane groups: sub-chunks per item (0: automatic);
                         // halo tiles: at most this many tiles per item (0: 4)
};

// One-thread-per-stage solve (tiled layout, n <= 32).
int tps_threads();
int tps_stages_per_subchunk();
size_t tps_smem_bytes(int nn_max, int precision);
cudaError_t tps_configure(int precision, size_t smem, int *blocks_per_sm);
cudaError_t launch_tps(const AdmmLaunch &a, int precision, cudaStream_t stream);

// Elementwise helpers.
cudaError_t launch_gather_n(const Layout &L, const double *xpart, const double *upart,
                            int64_t total_n, int precision, void *dst, cudaStream_t stream);
cudaError_t launch_gather_n64(const Layout &L, const double *xpart, const double *upart,
                              int64_t total_n, double *dst, cudaStream_t stream);
cudaError_t launch_convert(const double *src, int64_t count, int precision, void *dst,
                           cudaStream_t stream);
cudaError_t launch_export_iterates(const Layout &L, void *const *it, const int *base,
                                   int precision, double *z, double *v, double *th, double *be,
                                   double *la, cudaStream_t stream);

// Models.
int model_nparams(int model);
int model_dims(int model, int *nx, int *nu);
cudaError_t launch_linearise(const Layout &L, int model, const double *params, double dt,
                             const double *xbar, const double *ubar, double *A, double *B,
                             double *e, int64_t total_points, const int *pinst,
                             const int64_t *pbase, cudaStream_t stream);
cudaError_t launch_plant_step(const Layout &L, int model, const double *params, double dt,
                              const double *x, const double *u, double *x_next,
                              cudaStream_t stream);

}  // namespace pimpc

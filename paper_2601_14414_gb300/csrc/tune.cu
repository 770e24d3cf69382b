// tune.cu -- schedules of the batched solve and the autotuner that picks one by timing.
//
// A schedule fixes how the persistent solve cuts its work: the kernel family (lane groups on
// plain stage blocks, lane groups owning 4-column blocks on blocked stage blocks, one thread per
// stage on halo tiles, every instance resident in one CTA or a cluster, or dense contractions
// over blocks of stages for stage-invariant instances), the
// shared-memory budget of a CTA (CTAs per SM) and the item size. Changing the schedule changes the data layout, so the stage cache is rebuilt and the
// iterates restart from zero at the next solve. The autotuner times a fixed number of
// iterations of every candidate on the solver's own batch with CUDA events and keeps the
// fastest.
#include <cstring>
#include <string>
#include <vector>

#include "launch.h"
#include "pimpc.h"
#include "solver.h"

using namespace pimpc;

extern "C" {

int pimpc_set_schedule(pimpc_solver *s, int family, int ctas_per_sm, int item_scale) {
  if (!s) return PIMPC_EINVAL;
  cudaSetDevice(s->device);
  Schedule sc;
  sc.family = family;
  sc.ctas_per_sm = ctas_per_sm;
  sc.item_scale = item_scale;
  const Schedule old = s->sched;
  std::string why;
  const int rc = apply_schedule(s, sc, why);
  if (rc != PIMPC_OK) {
    std::string dummy;
    if (apply_schedule(s, old, dummy) != PIMPC_OK) why += " (and the previous schedule could not be restored)";
    return fail(s, rc, why);
  }
  return PIMPC_OK;
}

int pimpc_get_schedule(pimpc_solver *s, int *family, int *ctas_per_sm, int *item_scale,
                       int *grid, int *threads, int *items) {
  if (!s) return PIMPC_EINVAL;
  if (family) *family = s->sched.family;
  if (ctas_per_sm) *ctas_per_sm = s->sched.ctas_per_sm;
  if (item_scale) *item_scale = s->sched.item_scale;
  if (grid) *grid = s->grid_admm;
  if (threads) *threads = s->plan.threads;
  if (items) *items = s->nitems;
  return PIMPC_OK;
}

int pimpc_autotune(pimpc_solver *s, int trial_iters, int *family, int *ctas_per_sm,
                   int *item_scale, double *best_ms, void *stream) {
  if (!s) return PIMPC_EINVAL;
  if (trial_iters < 1) return fail(s, PIMPC_EINVAL, "trial_iters must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(s->device);
  std::vector<Schedule> cands;
  for (int m : {0, 2, 8}) {
    Schedule c;
    c.family = 0;
    c.item_scale = m;
    cands.push_back(c);
  }
  for (int cps : {2, 3, 4}) {
    Schedule c;
    c.family = 5;  // blocked lane groups, shared memory sized for cps CTAs per SM
    c.ctas_per_sm = cps;
    cands.push_back(c);
  }
  {
    Schedule c;
    c.family = 3;  // resident: skipped below when the instances do not fit
    cands.push_back(c);
  }
  if (s->lti) {
    Schedule c;
    c.family = 4;  // stage-invariant instances as dense contractions
    cands.push_back(c);
  }
  if (!s->accel) {
    Schedule c;
    c.family = 7;  // temporal blocking of the plain iteration
    cands.push_back(c);
  }
  if (s->lti && s->prec == PIMPC_F32) {
    Schedule c;
    c.family = 6;  // stage products on the tensor cores: skipped below when the sizes do not fit
    cands.push_back(c);
  }
  if (s->prec == PIMPC_F32 && !s->lti)
    for (int cps : {1, 2}) {
      Schedule c;
      c.family = 2;
      c.ctas_per_sm = cps;
      cands.push_back(c);
    }
  // Trial solves: zero state, no reference, a fixed number of iterations.
  const double eps = s->eps;
  const int max_iters = s->max_iters;
  const int stall_win = s->stall_win;
  const Schedule old = s->sched;
  s->eps = -1.0;
  s->max_iters = trial_iters;
  s->stall_win = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = -1.0;
  Schedule pick = old;
  int rc = PIMPC_OK;
  for (const Schedule &c : cands) {
    std::string why;
    if (apply_schedule(s, c, why) != PIMPC_OK) continue;  // this batch does not fit it
    cudaMemsetAsync(s->stage64, 0, sizeof(double) * s->tot_nx, st);
    rc = pimpc_factorise(s, stream);
    if (rc != PIMPC_OK) break;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == PIMPC_OK; ++rep) {
      cudaEventRecord(e0, st);
      rc = pimpc_solve(s, s->stage64, nullptr, nullptr, 0, 0, nullptr, nullptr, nullptr, nullptr,
                       nullptr, PIMPC_DEVICE, stream);
      cudaEventRecord(e1, st);
    }
    if (rc != PIMPC_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = cuda_fail(s, cudaGetLastError(), "autotune"); break; }
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.0 || ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->eps = eps;
  s->max_iters = max_iters;
  s->stall_win = stall_win;
  std::string why;
  const int rc2 = apply_schedule(s, rc == PIMPC_OK ? pick : old, why);
  if (rc != PIMPC_OK) return rc;
  if (rc2 != PIMPC_OK) return fail(s, rc2, why);
  if (family) *family = pick.family;
  if (ctas_per_sm) *ctas_per_sm = pick.ctas_per_sm;
  if (item_scale) *item_scale = pick.item_scale;
  if (best_ms) *best_ms = best;
  return PIMPC_OK;
}

}  // extern "C"

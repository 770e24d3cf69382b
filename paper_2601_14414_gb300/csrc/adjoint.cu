// adjoint.cu -- reverse mode of the unrolled iteration (work in progress).
#include "launch.h"
#include "pimpc.h"

extern "C" int pimpc_backward(pimpc_solver *s, const double *dL_du, const double *dL_dx,
                              double *g_x0, double *g_ref, double *g_q, double *g_r,
                              double *g_xmin, double *g_xmax, double *g_umin, double *g_umax,
                              int checkpoint_every, int mem, void *stream) {
  (void)s; (void)dL_du; (void)dL_dx; (void)g_x0; (void)g_ref; (void)g_q; (void)g_r;
  (void)g_xmin; (void)g_xmax; (void)g_umin; (void)g_umax; (void)checkpoint_every; (void)mem;
  (void)stream;
  return PIMPC_ESTATE;
}

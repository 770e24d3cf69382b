// noalloc.cu -- pimpc_solve_static: one MPC instance solved without any device allocation.
//
// Some callers cannot call cudaMalloc: real-time control loops that forbid allocation after
// start-up (an allocation can synchronise the device and has no latency bound), controllers
// certified without dynamic memory, and plug-ins inside a host whose device memory belongs to
// another framework's allocator. For them this entry point takes every input
// and output as device memory owned by the caller and keeps all of its own working memory
// (stage blocks, iterates, per-instance state, work list, control block) in one file-scope
// device array of fixed size, kStaticBytes. Every GPU that loads the library holds that array
// until the process exits.
//
// The array is shared by every call: calls that overlap on the GPU (on different streams, or
// from different host threads) race on it. Each call rewrites or clears everything it reads
// before reading it. The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device); make that first call before any stream capture.
//
// The arithmetic is that of pimpc_solve: the same factorisation, solve and output kernels run
// on the same memory layout, with their buffers carved out of the static array.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "launch.h"
#include "pimpc.h"

namespace pimpc {
void set_thread_error(const std::string &msg);
cudaError_t launch_unpack_state(const InstState *st, int batch, int *iters, double *c,
                                int *status, int *momentum, cudaStream_t stream);
}  // namespace pimpc

using namespace pimpc;

namespace {

constexpr size_t kStaticBytes = (size_t)16 << 20;  // 16 MiB, documented in include/pimpc.h
__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t rc = cudaGetDevice(&dev);
  if (rc != cudaSuccess) return rc;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    rc = cudaGetSymbolAddress(&p, g_static_scratch);
    if (rc != cudaSuccess) return rc;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carver {
  unsigned char *base;
  size_t used = 0;
  template <typename P>
  P *take(size_t count) {
    used = (used + 255) & ~(size_t)255;
    P *p = reinterpret_cast<P *>(base + used);
    used += count * sizeof(P);
    return p;
  }
};

struct Views {
  int *nx, *nu, *N, *W;
  int64_t *off[13];  // off_nx, off_nu, off_n, Nnx, Nnu, Nn, offA, offB, offe, blk, stage0, bbase, Ni
  int *binst, *item_inst, *item_a, *item_b, *nitems_inst, *list0, *list1;
  int *base, *old_base, *ndone, *stop, *ferr;
  double *alpha, *cprev, *coef, *cacc, *qd64;
  InstState *st;
  Ctl *ctl;
};

// Fills the single-instance layout and work list (all offsets 0, one instance).
__global__ void static_setup_kernel(Views v, int nx, int nu, int N, int W, int64_t Ni_total,
                                    int item_stages, int nitems) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    v.nx[0] = nx;
    v.nu[0] = nu;
    v.N[0] = N;
    v.W[0] = W;
    for (int i = 0; i < 13; ++i) v.off[i][0] = 0;
    v.base[0] = 0;
    v.nitems_inst[0] = nitems;
    v.ferr[0] = 0;
    (void)Ni_total;
  }
  for (int k = t; k < N; k += gridDim.x * blockDim.x) v.binst[k] = 0;
  for (int i = t; i < nitems; i += gridDim.x * blockDim.x) {
    v.item_inst[i] = 0;
    v.item_a[i] = i * item_stages;
    v.item_b[i] = min(N, (i + 1) * item_stages);
  }
}

int fail_static(int code, const std::string &msg) {
  set_thread_error(msg);
  return code;
}

}  // namespace

extern "C" int pimpc_solve_static(int nx, int nu, int N, int precision, const double *A,
                                  const double *B, const double *e, const double *q,
                                  const double *r, const double *xmin, const double *xmax,
                                  const double *umin, const double *umax, const double *x0,
                                  const double *ref, double rho, double eps, int max_iters,
                                  int accel, double eta, double *u_out, double *x_out,
                                  int *iters, double *c, int *status, void *stream) {
  const int n = nx + nu;
  if (nx < 1 || nu < 1 || N < 1 || n > PIMPC_MAX_N_LTV)
    return fail_static(PIMPC_EINVAL, "pimpc_solve_static: need nx >= 1, nu >= 1, N >= 1, nx + nu <= 32");
  if (precision != PIMPC_F32 && precision != PIMPC_F64)
    return fail_static(PIMPC_EINVAL, "pimpc_solve_static: bad precision");
  if (!A || !B || !q || !r || !xmin || !xmax || !umin || !umax || !x0)
    return fail_static(PIMPC_EINVAL, "pimpc_solve_static: missing input");
  // The same option checks as pimpc_set_options.
  if (!(rho > 0.0) || !std::isfinite(rho))
    return fail_static(PIMPC_EINVAL, "pimpc_solve_static: rho must be finite and > 0");
  if (std::isnan(eps)) return fail_static(PIMPC_EINVAL, "pimpc_solve_static: eps is NaN");
  if (max_iters < 0) return fail_static(PIMPC_EINVAL, "pimpc_solve_static: max_iters < 0");
  if (accel != 0 && accel != 1)
    return fail_static(PIMPC_EINVAL, "pimpc_solve_static: accel must be 0 or 1");
  if (!(eta >= 0.0) || !std::isfinite(eta))
    return fail_static(PIMPC_EINVAL, "pimpc_solve_static: eta must be finite and >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ts = precision == PIMPC_F32 ? 4 : 8;
  const int64_t ntiles = (N + 31) / 32;
  const int W = nx * n + nx + n * (n + 1) / 2 + nu * (nu + 1) / 2;
  const int64_t blk_elems = (ntiles * 32 * W + 31) / 32 * 32;
  const int64_t it_elems = ntiles * 32 * 5 * n;
  const int S = tps_stages_per_subchunk();
  const int item_stages = S;
  const int nitems = (N + item_stages - 1) / item_stages;

  void *raw = nullptr;
  cudaError_t rc = scratch_address(&raw);
  if (rc != cudaSuccess)
    return fail_static(PIMPC_ECUDA, std::string("pimpc_solve_static: cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(rc));
  Carver cv{(unsigned char *)raw};
  Views v;
  v.nx = cv.take<int>(1); v.nu = cv.take<int>(1); v.N = cv.take<int>(1); v.W = cv.take<int>(1);
  for (int i = 0; i < 13; ++i) v.off[i] = cv.take<int64_t>(1);
  v.binst = cv.take<int>(N);
  v.item_inst = cv.take<int>(nitems); v.item_a = cv.take<int>(nitems); v.item_b = cv.take<int>(nitems);
  v.nitems_inst = cv.take<int>(1);
  v.list0 = cv.take<int>(nitems); v.list1 = cv.take<int>(nitems);
  v.base = cv.take<int>(1); v.old_base = cv.take<int>(1); v.ndone = cv.take<int>(1);
  v.stop = cv.take<int>(1); v.ferr = cv.take<int>(1);
  v.alpha = cv.take<double>(1); v.cprev = cv.take<double>(1); v.coef = cv.take<double>(1);
  v.cacc = cv.take<double>(1); v.qd64 = cv.take<double>(n);
  v.st = cv.take<InstState>(1);
  v.ctl = cv.take<Ctl>(1);
  unsigned char *blk = cv.take<unsigned char>(blk_elems * ts);
  unsigned char *its[3];
  for (int b = 0; b < 3; ++b) its[b] = cv.take<unsigned char>(it_elems * ts);
  unsigned char *qd_T = cv.take<unsigned char>(n * ts), *ref_T = cv.take<unsigned char>(n * ts);
  unsigned char *lo_T = cv.take<unsigned char>(n * ts), *hi_T = cv.take<unsigned char>(n * ts);
  unsigned char *xb0_T = cv.take<unsigned char>(n * ts);
  if (cv.used > kStaticBytes) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "pimpc_solve_static: this instance needs %zu bytes of working memory, more than the "
             "%zu-byte static array",
             cv.used, kStaticBytes);
    return fail_static(PIMPC_EINVAL, msg);
  }

  Layout L{};
  L.batch = 1; L.lti = 0; L.tiled = 1;
  L.nx = v.nx; L.nu = v.nu; L.N = v.N; L.W = v.W;
  L.off_nx = v.off[0]; L.off_nu = v.off[1]; L.off_n = v.off[2];
  L.Nnx = v.off[3]; L.Nnu = v.off[4]; L.Nn = v.off[5];
  L.offA = v.off[6]; L.offB = v.off[7]; L.offe = v.off[8];
  L.blk = v.off[9]; L.stage0 = v.off[10]; L.Ni = v.off[12];

  auto check = [&](cudaError_t e2, const char *what) -> int {
    if (e2 == cudaSuccess) return PIMPC_OK;
    return fail_static(PIMPC_ECUDA, std::string("pimpc_solve_static: ") + what + ": " +
                                        cudaGetErrorString(e2));
  };
  int ret;
  static_setup_kernel<<<1, 128, 0, st>>>(v, nx, nu, N, W, it_elems, item_stages, nitems);
  if ((ret = check(cudaGetLastError(), "setup"))) return ret;
  // Everything the kernels read before writing starts from a known state on every call.
  if ((ret = check(cudaMemsetAsync(blk, 0, blk_elems * ts, st), "clear stage blocks"))) return ret;
  if ((ret = check(launch_gather_n64(L, q, r, n, v.qd64, st), "weights"))) return ret;
  if ((ret = check(launch_gather_n(L, q, r, n, precision, qd_T, st), "weights"))) return ret;
  if ((ret = check(launch_gather_n(L, xmin, umin, n, precision, lo_T, st), "bounds"))) return ret;
  if ((ret = check(launch_gather_n(L, xmax, umax, n, precision, hi_T, st), "bounds"))) return ret;
  if ((ret = check(launch_gather_n(L, x0, nullptr, n, precision, xb0_T, st), "x0"))) return ret;
  if (ref && (ret = check(launch_convert(ref, n, precision, ref_T, st), "ref"))) return ret;
  if ((ret = check(launch_factorise(L, A, B, e, v.qd64, nullptr, rho, v.binst, v.off[11], N, nx, n,
                                    precision, blk, v.ferr, st), "factorise")))
    return ret;

  AdmmLaunch a{};
  a.L = L;
  a.blk = blk;
  for (int b = 0; b < 3; ++b) a.it[b] = its[b];
  a.qd = qd_T; a.ref = ref ? ref_T : nullptr; a.ref_per_stage = 0;
  a.lo = lo_T; a.hi = hi_T; a.xb0 = xb0_T;
  a.rho = rho; a.eps = eps; a.eta = eta; a.max_iters = max_iters; a.accel = accel;
  a.mask = nullptr; a.mask_len = 0;
  a.item_inst = v.item_inst; a.item_a = v.item_a; a.item_b = v.item_b;
  a.nitems_inst = v.nitems_inst; a.nitems = nitems;
  a.list0 = v.list0; a.list1 = v.list1; a.ctl = v.ctl;
  a.base = v.base; a.old_base = v.old_base; a.st = v.st;
  a.alpha = v.alpha; a.cprev = v.cprev; a.coef = v.coef; a.cacc = v.cacc;
  a.ndone = v.ndone; a.stop = v.stop;
  a.u_out = u_out; a.x_out = x_out;
  a.warm = 0;  // cold start: the iterate buffer is cleared by the launch sequence
  a.ferr = v.ferr;
  a.threads = tps_threads();
  a.nv_max = n;
  const size_t smem = tps_smem_bytes(n, precision);
  int bps = 0, nsm = 0, dev = 0;
  if ((ret = check(tps_configure(precision, smem, &bps), "configure"))) return ret;
  if ((ret = check(cudaGetDevice(&dev), "device"))) return ret;
  if ((ret = check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "device"))) return ret;
  a.grid = std::min(nitems, std::max(1, bps * nsm));
  if ((ret = check(launch_tps(a, precision, st), "solve"))) return ret;
  if (iters || c || status)
    if ((ret = check(launch_unpack_state(v.st, 1, iters, c, status, nullptr, st), "results"))) return ret;
  return PIMPC_OK;
}

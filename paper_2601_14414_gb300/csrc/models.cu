// models.cu -- built-in nonlinear models, explicit-Euler relinearisation and the plant step.
//
// Real-time iteration (the NMPC scheme the paper's LTV formulation generalises, Sec. I-II): at
// every sample the model x_{k+1} = F(x_k, u_k) = x_k + dt f(x_k, u_k) is linearised along a
// trajectory, A_k = dF/dx, B_k = dF/du, e_k = F(xbar_k, ubar_k) - A_k xbar_k - B_k ubar_k,
// and the solver runs on the resulting stage matrices without building a QP. Jacobians come
// from forward-mode dual numbers, one seed direction at a time, all in FP64; one thread per
// linearisation point.
#include <math.h>

#include "launch.h"

namespace pimpc {

namespace {

// First-order dual number v + d eps.
struct Dual {
  double v, d;
  __device__ Dual() {}
  __device__ Dual(double a, double b = 0.0) : v(a), d(b) {}
};
__device__ inline Dual mk(double v, double d) { return Dual(v, d); }
__device__ inline Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
__device__ inline Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
__device__ inline Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ inline Dual operator/(Dual a, Dual b) {
  return Dual{a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
__device__ inline Dual operator*(double s, Dual a) { return Dual{s * a.v, s * a.d}; }
__device__ inline Dual operator+(double s, Dual a) { return Dual{s + a.v, a.d}; }
__device__ inline Dual operator-(double s, Dual a) { return Dual{s - a.v, -a.d}; }
__device__ inline Dual sin(Dual a) { return Dual{::sin(a.v), ::cos(a.v) * a.d}; }
__device__ inline Dual cos(Dual a) { return Dual{::cos(a.v), -::sin(a.v) * a.d}; }
__device__ inline Dual exp(Dual a) {
  double e = ::exp(a.v);
  return Dual{e, e * a.d};
}

__device__ inline double dsin(double a) { return ::sin(a); }
__device__ inline double dcos(double a) { return ::cos(a); }
__device__ inline double dexp(double a) { return ::exp(a); }
__device__ inline Dual dsin(Dual a) { return sin(a); }
__device__ inline Dual dcos(Dual a) { return cos(a); }
__device__ inline Dual dexp(Dual a) { return exp(a); }

// Quadrotor, "+" layout: x = (position, velocity, roll, pitch, yaw, body rates), u = rotor
// thrusts; p = (m, g, Jx, Jy, Jz, arm, yaw coefficient). Rotation R = Rz(yaw) Ry(pitch) Rx(roll).
template <typename S>
__device__ void quadrotor(const double *p, const S *x, const S *u, S *f) {
  const double m = p[0], g = p[1], Jx = p[2], Jy = p[3], Jz = p[4], arm = p[5], kq = p[6];
  const S thrust = u[0] + u[1] + u[2] + u[3];
  const S tau_x = arm * (u[1] - u[3]);
  const S tau_y = arm * (u[2] - u[0]);
  const S tau_z = kq * ((u[0] + u[2]) - (u[1] + u[3]));
  const S sr = dsin(x[6]), cr = dcos(x[6]);
  const S sp = dsin(x[7]), cp = dcos(x[7]);
  const S sy = dsin(x[8]), cy = dcos(x[8]);
  const S wx = x[9], wy = x[10], wz = x[11];
  const S acc = (1.0 / m) * thrust;
  for (int i = 0; i < 3; ++i) f[i] = x[3 + i];
  f[3] = acc * (cy * sp * cr + sy * sr);
  f[4] = acc * (sy * sp * cr - cy * sr);
  f[5] = acc * (cp * cr) - S(g);
  // roll/pitch/yaw rates from body rates
  f[6] = wx + (sr * wy + cr * wz) * (sp / cp);
  f[7] = cr * wy - sr * wz;
  f[8] = (sr * wy + cr * wz) / cp;
  // J dw/dt = tau - w x (J w), J diagonal
  f[9] = (1.0 / Jx) * (tau_x - (Jz - Jy) * (wy * wz));
  f[10] = (1.0 / Jy) * (tau_y - (Jx - Jz) * (wz * wx));
  f[11] = (1.0 / Jz) * (tau_z - (Jy - Jx) * (wx * wy));
}

// Cart-pole with a uniform pole (half-length l), upright at angle 0:
// x = (cart position, cart velocity, angle, angular rate), u = force; p = (mc, mp, l, g).
template <typename S>
__device__ void cartpole(const double *p, const S *x, const S *u, S *f) {
  const double mc = p[0], mp = p[1], l = p[2], g = p[3], mt = mc + mp;
  const S s = dsin(x[2]), c = dcos(x[2]);
  const S w = x[3];
  const S b = (1.0 / mt) * (u[0] + (mp * l) * (w * w) * s);
  const S ang = (g * s - c * b) / (l * (4.0 / 3.0 - (mp / mt) * (c * c)));
  f[0] = x[1];
  f[1] = b - ((mp * l) / mt) * (ang * c);
  f[2] = w;
  f[3] = ang;
}

// CSTR of the paper's example (Sec. V): x = (C_A, T), u = T_c; p = (C_Ai, k0, EaR, T_i).
template <typename S>
__device__ void cstr(const double *p, const S *x, const S *u, S *f) {
  const S rate = p[1] * (dexp(-p[2] / x[1]) * x[0]);
  f[0] = (p[0] - x[0]) - rate;
  f[1] = (p[3] + 0.3 * u[0]) - 1.3 * x[1] + 11.92 * rate;
}

template <typename S>
__device__ void eval_model(int model, const double *p, const S *x, const S *u, S *f) {
  if (model == 0) quadrotor(p, x, u, f);
  else if (model == 1) cartpole(p, x, u, f);
  else cstr(p, x, u, f);
}

__device__ __host__ inline int nparams(int model) { return model == 0 ? 7 : 4; }

constexpr int kMaxModelDim = 16;

// One thread per linearisation point (stage k of instance j, or instance j for LTI data).
__global__ void linearise_kernel(Layout L, int model, const double *params, double dt,
                                 const double *xbar, const double *ubar, double *A, double *B,
                                 double *e, int64_t total, const int *pinst,
                                 const int64_t *pbase) {
  const int64_t pt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= total) return;
  const int j = pinst ? pinst[pt] : (int)pt;
  const int k = pinst ? (int)(pt - pbase[j]) : 0;
  const int nx = L.nx[j], nu = L.nu[j];
  const double *p = params + (int64_t)j * nparams(model);
  const int64_t sx = (L.lti ? L.off_nx[j] : L.Nnx[j]) + (int64_t)k * nx;
  const int64_t su = (L.lti ? L.off_nu[j] : L.Nnu[j]) + (int64_t)k * nu;
  double xv[kMaxModelDim], uv[kMaxModelDim], f0[kMaxModelDim];
  for (int i = 0; i < nx; ++i) xv[i] = xbar[sx + i];
  for (int i = 0; i < nu; ++i) uv[i] = ubar[su + i];
  eval_model(model, p, xv, uv, f0);
  double *Ak = A + L.offA[j] + (int64_t)k * nx * nx;
  double *Bk = B + L.offB[j] + (int64_t)k * nx * nu;
  double *ek = e + L.offe[j] + (int64_t)k * nx;
  Dual xd[kMaxModelDim], ud[kMaxModelDim], fd[kMaxModelDim];
  for (int dir = 0; dir < nx + nu; ++dir) {
    for (int i = 0; i < nx; ++i) xd[i] = mk(xv[i], i == dir ? 1.0 : 0.0);
    for (int i = 0; i < nu; ++i) ud[i] = mk(uv[i], nx + i == dir ? 1.0 : 0.0);
    eval_model(model, p, xd, ud, fd);
    for (int i = 0; i < nx; ++i) {
      if (dir < nx) Ak[i * nx + dir] = (i == dir ? 1.0 : 0.0) + dt * fd[i].d;
      else Bk[i * nu + (dir - nx)] = dt * fd[i].d;
    }
  }
  for (int i = 0; i < nx; ++i) {
    double s = xv[i] + dt * f0[i];
    for (int c = 0; c < nx; ++c) s -= Ak[i * nx + c] * xv[c];
    for (int c = 0; c < nu; ++c) s -= Bk[i * nu + c] * uv[c];
    ek[i] = s;
  }
}

__global__ void plant_kernel(Layout L, int model, const double *params, double dt, const double *x,
                             const double *u, double *x_next) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L.batch) return;
  const int nx = L.nx[j], nu = L.nu[j];
  double xv[kMaxModelDim], uv[kMaxModelDim], f[kMaxModelDim];
  for (int i = 0; i < nx; ++i) xv[i] = x[L.off_nx[j] + i];
  for (int i = 0; i < nu; ++i) uv[i] = u[L.off_nu[j] + i];
  eval_model(model, params + (int64_t)j * nparams(model), xv, uv, f);
  for (int i = 0; i < nx; ++i) x_next[L.off_nx[j] + i] = xv[i] + dt * f[i];
}

}  // namespace

int model_nparams(int model) { return nparams(model); }

int model_dims(int model, int *nx, int *nu) {
  switch (model) {
    case 0: *nx = 12; *nu = 4; return 0;
    case 1: *nx = 4; *nu = 1; return 0;
    case 2: *nx = 2; *nu = 1; return 0;
    default: return -1;
  }
}

cudaError_t launch_linearise(const Layout &L, int model, const double *params, double dt,
                             const double *xbar, const double *ubar, double *A, double *B,
                             double *e, int64_t total_points, const int *pinst,
                             const int64_t *pbase, cudaStream_t stream) {
  if (total_points == 0) return cudaSuccess;
  const int threads = 128;
  const int64_t grid = (total_points + threads - 1) / threads;
  linearise_kernel<<<(unsigned)grid, threads, 0, stream>>>(L, model, params, dt, xbar, ubar, A, B,
                                                           e, total_points, pinst, pbase);
  return cudaGetLastError();
}

cudaError_t launch_plant_step(const Layout &L, int model, const double *params, double dt,
                              const double *x, const double *u, double *x_next,
                              cudaStream_t stream) {
  const int threads = 128;
  plant_kernel<<<(L.batch + threads - 1) / threads, threads, 0, stream>>>(L, model, params, dt, x,
                                                                          u, x_next);
  return cudaGetLastError();
}

}  // namespace pimpc

// misc.cu -- elementwise marshalling kernels: FP64 ABI arrays <-> the solver's internal layout.
#include "lockstep.cuh"

namespace pimpc {

namespace {

// dst[off_n[j] + c] = c < nx ? xpart[off_nx[j] + c] : upart[off_nu[j] + c - nx]; one block per
// instance, upart == null gives 0 for the input part.
template <typename T>
__global__ void gather_n_kernel(Layout L, const double *xpart, const double *upart, T *dst) {
  const int j = blockIdx.x;
  const int nx = L.nx[j], nu = L.nu[j], n = nx + nu;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double v;
    if (c < nx) v = xpart ? xpart[L.off_nx[j] + c] : 0.0;
    else v = upart ? upart[L.off_nu[j] + c - nx] : 0.0;
    dst[L.off_n[j] + c] = (T)v;
  }
}

template <typename T>
__global__ void convert_kernel(const double *src, int64_t count, T *dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

// Iterates of stage k (vectors z, v, theta, beta, lambda in either layout) -> five [sum N n]
// FP64 arrays.
template <typename T>
__global__ void export_kernel(Layout L, T *it0, T *it1, T *it2, const int *base, double *z,
                              double *v, double *th, double *be, double *la) {
  const int j = blockIdx.x;
  const int n = L.nx[j] + L.nu[j], N = L.N[j];
  const int n5p = ls::iter_stride_plain(n, (int)sizeof(T));
  T *bufs[3] = {it0, it1, it2};
  const T *src = bufs[base[j]] + L.Ni[j];
  double *outs[5] = {z, v, th, be, la};
  const int tw = ls::layout_aux(L, j);
  for (int64_t t = threadIdx.x; t < (int64_t)N * n; t += blockDim.x) {
    const int k = (int)(t / n), c = (int)(t - (int64_t)k * n);
    for (int b = 0; b < 5; ++b)
      if (outs[b])
        outs[b][L.Nn[j] + t] = (double)src[ls::iter_index(L.tiled, tw, n, n5p, k, b, c)];
  }
}

}  // namespace

cudaError_t launch_gather_n(const Layout &L, const double *xpart, const double *upart,
                            int64_t total_n, int precision, void *dst, cudaStream_t stream) {
  (void)total_n;
  if (precision == 0)
    gather_n_kernel<float><<<L.batch, 64, 0, stream>>>(L, xpart, upart, (float *)dst);
  else
    gather_n_kernel<double><<<L.batch, 64, 0, stream>>>(L, xpart, upart, (double *)dst);
  return cudaGetLastError();
}

cudaError_t launch_gather_n64(const Layout &L, const double *xpart, const double *upart,
                              int64_t total_n, double *dst, cudaStream_t stream) {
  (void)total_n;
  gather_n_kernel<double><<<L.batch, 64, 0, stream>>>(L, xpart, upart, dst);
  return cudaGetLastError();
}

cudaError_t launch_convert(const double *src, int64_t count, int precision, void *dst,
                           cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (precision == 0)
    convert_kernel<float><<<(unsigned)blocks, 256, 0, stream>>>(src, count, (float *)dst);
  else
    convert_kernel<double><<<(unsigned)blocks, 256, 0, stream>>>(src, count, (double *)dst);
  return cudaGetLastError();
}

cudaError_t launch_export_iterates(const Layout &L, void *const *it, const int *base,
                                   int precision, double *z, double *v, double *th, double *be,
                                   double *la, cudaStream_t stream) {
  if (precision == 0)
    export_kernel<float><<<L.batch, 256, 0, stream>>>(L, (float *)it[0], (float *)it[1],
                                                      (float *)it[2], base, z, v, th, be, la);
  else
    export_kernel<double><<<L.batch, 256, 0, stream>>>(L, (double *)it[0], (double *)it[1],
                                                       (double *)it[2], base, z, v, th, be, la);
  return cudaGetLastError();
}

}  // namespace pimpc

namespace pimpc {

namespace {

__global__ void unpack_state_kernel(const InstState *st, int batch, int *iters, double *c,
                                    int *status, int *momentum) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  if (iters) iters[j] = st[j].iters;
  if (c) c[j] = st[j].c;
  if (status) status[j] = st[j].status;
  if (momentum) momentum[j] = st[j].momentum;
}

// Iterates of the latest buffer of one layout (iteration type S) -> the latest buffer of a
// plain FP64 layout (the polish's starting point); one block per instance.
template <typename S>
__global__ void copy_iterates_kernel(Layout Ls, const S *s0, const S *s1, const S *s2,
                                     const int *base_s, Layout Ld, double *d0, double *d1,
                                     double *d2, const int *base_d) {
  const int j = blockIdx.x;
  const int n = Ls.nx[j] + Ls.nu[j], N = Ls.N[j];
  const S *srcs[3] = {s0, s1, s2};
  double *dsts[3] = {d0, d1, d2};
  const S *src = srcs[base_s[j]] + Ls.Ni[j];
  double *dst = dsts[base_d[j]] + Ld.Ni[j];
  const int n5s = ls::iter_stride_plain(n, (int)sizeof(S)), n5d = ls::iter_stride_plain(n, 8);
  const int tws = ls::layout_aux(Ls, j);
  for (int64_t t = threadIdx.x; t < (int64_t)N * 5 * n; t += blockDim.x) {
    const int k = (int)(t / (5 * n)), r = (int)(t - (int64_t)k * 5 * n);
    const int b = r / n, c = r - b * n;
    dst[ls::iter_index(Ld.tiled, 0, n, n5d, k, b, c)] =
        (double)src[ls::iter_index(Ls.tiled, tws, n, n5s, k, b, c)];
  }
}

__global__ void add_state_kernel(InstState *st, const InstState *polish, int batch) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  st[j].iters += polish[j].iters;
  st[j].momentum += polish[j].momentum;
  st[j].c = polish[j].c;
  st[j].status = polish[j].status;
}

__global__ void fill_kernel(double *dst, int64_t count, double value) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = value;
}

}  // namespace

cudaError_t launch_unpack_state(const InstState *st, int batch, int *iters, double *c,
                                int *status, int *momentum, cudaStream_t stream) {
  unpack_state_kernel<<<(batch + 127) / 128, 128, 0, stream>>>(st, batch, iters, c, status,
                                                               momentum);
  return cudaGetLastError();
}

cudaError_t launch_copy_iterates(const Layout &Ls, void *const *its, const int *base_s, int prec_s,
                                 const Layout &Ld, void *const *itd, const int *base_d,
                                 cudaStream_t stream) {
  double *const *d = reinterpret_cast<double *const *>(itd);
  if (prec_s == 0)
    copy_iterates_kernel<float><<<Ls.batch, 256, 0, stream>>>(
        Ls, (const float *)its[0], (const float *)its[1], (const float *)its[2], base_s, Ld, d[0],
        d[1], d[2], base_d);
  else
    copy_iterates_kernel<double><<<Ls.batch, 256, 0, stream>>>(
        Ls, (const double *)its[0], (const double *)its[1], (const double *)its[2], base_s, Ld,
        d[0], d[1], d[2], base_d);
  return cudaGetLastError();
}

cudaError_t launch_add_state(InstState *st, const InstState *polish, int batch, cudaStream_t stream) {
  add_state_kernel<<<(batch + 127) / 128, 128, 0, stream>>>(st, polish, batch);
  return cudaGetLastError();
}

cudaError_t launch_fill(double *dst, int64_t count, double value, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  fill_kernel<<<(unsigned)blocks, 256, 0, stream>>>(dst, count, value);
  return cudaGetLastError();
}

}  // namespace pimpc

// usets.cuh -- Euclidean projection of the input part of z_{k+1} onto a non-box convex set
// (internal).
//
// The remark after Theorem 1: the reduced (v, z) problem of the splitting has the Hessian (3/2) I
// whatever the constraint set, so z_{k+1} stays the Euclidean projection of the same point w
// (Algorithm 1 step 2). The state part keeps its box; the input part u = w[nx:n] is projected
// onto one of
//   kUsetBall2      ||u||_2 <= r            u min(1, r / ||u||)
//   kUsetBall1      ||u||_1 <= r            soft threshold at tau, sum max(|u_i| - tau, 0) = r
//   kUsetHalfspace  a^T u <= r              u - max(0, a^T u - r) / ||a||^2 a
//   kUsetSoc        ||u_{1:}||_2 <= u_0     the second-order cone
// The n components of a stage are spread over the g lanes of a group (g a power of two, groups
// aligned inside the warp); each lane holds K of them. All 32 lanes of the warp call these
// functions together (uniform control flow; a lane without a stage passes no valid component):
// the group's sums are butterfly reductions with offsets below g.
#pragma once

namespace pimpc {
namespace uset {

constexpr int kUsetBox = 0, kUsetBall2 = 1, kUsetBall1 = 2, kUsetHalfspace = 3, kUsetSoc = 4;

template <typename T>
__device__ __forceinline__ T group_sum(T v, int g) {
  for (int off = g >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename T>
__device__ __forceinline__ T group_max(T v, int g) {
  for (int off = g >> 1; off > 0; off >>= 1) {
    const T o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}

// Value of slot s of lane `src` (all lanes pass the same s).
template <typename T, int K>
__device__ __forceinline__ T fetch(const T (&v)[K], int s, int src) {
  T mine = v[0];
#pragma unroll
  for (int q = 1; q < K; ++q)
    if (s == q) mine = v[q];
  return __shfl_sync(0xffffffffu, mine, src);
}

// Projects w[q] for the owned components c[q] (c[q] < 0: none) with nx <= c[q] < n onto the set
// `kind` (1..4), in place; state components are left alone. Layout: component j lives in lane
// `lane_of(j)` of the group, slot `slot_of(j)`. a[q] is the halfspace normal of component c[q].
template <typename T, int K, typename LaneOf, typename SlotOf>
__device__ void project_inputs(int kind, T r, const T (&a)[K], T (&w)[K], const int (&c)[K], int nx,
                               int n, int g, LaneOf lane_of, SlotOf slot_of) {
  const int base = (threadIdx.x & 31) & ~(g - 1);
  bool in[K];
#pragma unroll
  for (int q = 0; q < K; ++q) in[q] = c[q] >= nx && c[q] < n;
  if (kind == kUsetBall2) {
    T s = (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q) if (in[q]) s += w[q] * w[q];
    const T nrm = sqrt(group_sum(s, g));
    const T f = nrm <= r ? (T)1 : r / nrm;
#pragma unroll
    for (int q = 0; q < K; ++q) if (in[q]) w[q] *= f;
  } else if (kind == kUsetHalfspace) {
    T s1 = (T)0, s2 = (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (in[q]) {
        s1 += a[q] * w[q];
        s2 += a[q] * a[q];
      }
    s1 = group_sum(s1, g);
    s2 = group_sum(s2, g);
    const T f = s1 > r ? (s1 - r) / s2 : (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q) if (in[q]) w[q] -= f * a[q];
  } else if (kind == kUsetSoc) {
    const T t = fetch<T, K>(w, slot_of(nx), base + lane_of(nx));
    T s = (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q) if (in[q] && c[q] > nx) s += w[q] * w[q];
    const T ns = sqrt(group_sum(s, g));
    if (ns <= t) return;
    if (ns <= -t) {
#pragma unroll
      for (int q = 0; q < K; ++q) if (in[q]) w[q] = (T)0;
      return;
    }
    const T al = (T)0.5 * (t + ns);
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (in[q]) w[q] = c[q] == nx ? al : al * w[q] / ns;
  } else if (kind == kUsetBall1) {
    T av[K];
    T tot = (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      av[q] = in[q] ? fabs(w[q]) : (T)0;
      tot += av[q];
    }
    const bool inside = group_sum(tot, g) <= r;  // no return here: the shuffles below are warp-wide
    // Sort-free threshold: for an input i with a_i = |u_i|, let cnt_i and s_i be the count and
    // the sum of the a_j >= a_i. The support of the projection is the set of i with
    // a_i cnt_i > s_i - r, and tau = (s_i - r) / cnt_i for the support member of largest cnt_i.
    T cnt[K], sum[K];
#pragma unroll
    for (int q = 0; q < K; ++q) cnt[q] = sum[q] = (T)0;
    for (int j = nx; j < n; ++j) {
      const T aj = fetch<T, K>(av, slot_of(j), base + lane_of(j));
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (in[q] && aj >= av[q]) {
          cnt[q] += (T)1;
          sum[q] += aj;
        }
    }
    T key = (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (in[q] && av[q] * cnt[q] > sum[q] - r && cnt[q] > key) key = cnt[q];
    const T kmax = group_max(key, g);
    T tc = (T)0;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (in[q] && cnt[q] == kmax && av[q] * cnt[q] > sum[q] - r) tc = (sum[q] - r) / cnt[q];
    const T tau = group_max(tc, g);
    if (inside) return;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (in[q]) {
        const T m = av[q] - tau;
        w[q] = m > (T)0 ? copysign(m, w[q]) : (T)0;
      }
  }
}

}  // namespace uset
}  // namespace pimpc

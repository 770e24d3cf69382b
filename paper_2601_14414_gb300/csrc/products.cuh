// products.cuh -- per-stage matrix-vector products of the lane-group solve kernels (internal):
// one lane per output component, operands in shared memory.
#pragma once
#include <cuda_runtime.h>

namespace pimpc {

// (S x)_c for a symmetric m x m matrix S stored as wrapped diagonals: row d (d <= m/2) holds
// S[c][(c + d) mod m]; S[c][(c - d) mod m] = S[(c - d) mod m][c] is entry (c - d) mod m of row d.
// Consecutive lanes read consecutive words of each row and distinct words of x.
template <typename T>
__device__ __forceinline__ T sym_wrapped(const T *D, const T *x, int m, int c) {
  T acc0 = D[c] * x[c], acc1 = (T)0;
  const int half = (m - 1) / 2;
  int ip = c, im = c;
  const T *row = D;
  for (int d = 1; d <= half; ++d) {
    row += m;
    ip = (ip + 1 == m) ? 0 : ip + 1;
    im = (im == 0) ? m - 1 : im - 1;
    acc0 += row[c] * x[ip];
    acc1 += row[im] * x[im];
  }
  if ((m & 1) == 0) {
    row += m;
    const int jm = c + m / 2 < m ? c + m / 2 : c - m / 2;
    acc0 += row[c] * x[jm];
  }
  return acc0 + acc1;
}

// sum_{r < cnt} M[r * ld] * v[r] with v 16-byte aligned in shared memory (read as vectors,
// identical for every lane of the group, so the reads broadcast).
template <typename T>
__device__ __forceinline__ T dot_col(const T *M, int ld, const T *v, int cnt) {
  T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
  int r = 0;
  if constexpr (sizeof(T) == 4) {
    for (; r + 3 < cnt; r += 4) {
      const float4 q = *reinterpret_cast<const float4 *>(v + r);
      a0 += M[(r + 0) * ld] * q.x;
      a1 += M[(r + 1) * ld] * q.y;
      a2 += M[(r + 2) * ld] * q.z;
      a3 += M[(r + 3) * ld] * q.w;
    }
  } else {
    for (; r + 3 < cnt; r += 4) {
      const double2 q0 = *reinterpret_cast<const double2 *>(v + r);
      const double2 q1 = *reinterpret_cast<const double2 *>(v + r + 2);
      a0 += M[(r + 0) * ld] * q0.x;
      a1 += M[(r + 1) * ld] * q0.y;
      a2 += M[(r + 2) * ld] * q1.x;
      a3 += M[(r + 3) * ld] * q1.y;
    }
  }
  for (; r < cnt; ++r) a0 += M[r * ld] * v[r];
  return (a0 + a1) + (a2 + a3);
}

}  // namespace pimpc

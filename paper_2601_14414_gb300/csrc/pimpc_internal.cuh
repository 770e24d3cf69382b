// pimpc_internal.cuh -- device-side data layout shared by the library's CUDA sources.
//
// Batch layout. Instances are concatenated. For instance j with sizes (nx, nu, N), n = nx + nu:
//   user-facing arrays (FP64, the C ABI): per-instance vectors at off_nx[j] / off_nu[j] / off_n[j],
//   per-stage arrays at Nnx[j] = sum_{i<j} N_i nx_i, Nnu[j], Nn[j] = sum N_i n_i, matrices at
//   offA[j] (sum N nx^2, or sum nx^2 when lti), offB[j], offe[j].
//
// Stage block (iteration precision T), the unit the solve kernels stream. Plain layout (lane-group
// kernel): [ G_k = [A_k | B_k] : nx rows of stride odd_ld(n) ][ e_k : nx ][ H_k wrapped
// diagonals ][ M_k wrapped diagonals ], padded to a multiple of 4 elements (W words); an LTV
// instance has N blocks at blk[j] + k W, an LTI instance two (H_k for k < N-1, then H_{N-1}).
// Tiled layout (one-thread-per-stage kernel): see admm_tps.cu.
//
// Iterates (T): three rotating buffers it[0..2]; stage k of instance j holds [z | v | theta | beta |
// lambda] (5 n values, z = z_{k+1}, padded to a 16-byte multiple n5p) at Ni[j] + n5p k. base[j]
// names the buffer with the latest non-hat iterate after a solve.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pimpc {

constexpr int kConverged = 0;   // per-instance status codes (same values as the C ABI)
constexpr int kMaxIter = 1;
constexpr int kNonFinite = 2;
constexpr int kTimeout = 3;
constexpr int kMaxNLtv = 32;
constexpr int kMaxNLti = 64;

struct Layout {
  int batch;
  int lti;
  int tiled;                       // 1: 32-stage tiled layout (n <= 32); 0: plain stage-major
  const int *nx, *nu, *N;          // [batch]
  const int64_t *off_nx, *off_nu, *off_n;   // per-instance vector offsets
  const int64_t *Nnx, *Nnu, *Nn;   // per-stage array offsets
  const int64_t *offA, *offB, *offe;
  const int64_t *blk;              // stage-block offsets (elements of T)
  const int *W;                    // stage-block size (elements)
  const int64_t *stage0;           // global index of the instance's first stage
  const int64_t *Ni;               // iterate offsets: sum_{i<j} N_i n5p_i
};

// Control block of one persistent solve launch.
struct Ctl {
  int queue[2];          // item queue counters (alternating iterations)
  unsigned bar_count;    // grid barrier: arrivals and generation
  unsigned bar_gen;
  int active;            // instances still iterating
  int stopped;           // some instance stopped in this iteration
  int err;               // nonzero: a bounded wait timed out
  int nlist[2];          // lengths of the two active-item lists
  int pad[7];
};

__host__ __device__ inline int packed_size(int n) { return n * (n + 1) / 2; }
// Plain stage block of the lane-group kernel: G rows padded to an odd stride, symmetric H and M
// as wrapped diagonals (see wrapped_size).
__host__ __device__ inline int odd_ld(int n) { return n | 1; }
// Wrapped-diagonal storage of a symmetric m x m matrix S: for d = 0 .. m/2, row d holds
// S[c][(c + d) mod m] for c = 0 .. m-1. Diagonals d and m-d hold the same elements, so only
// d <= m/2 is stored: m (1 + floor((m-1)/2) + [m even]) elements.
__host__ __device__ inline int wrapped_rows(int m) { return 1 + (m - 1) / 2 + ((m % 2 == 0) ? 1 : 0); }
__host__ __device__ inline int wrapped_size(int m) { return m * wrapped_rows(m); }
__host__ __device__ inline int block_words(int nx, int nu) {
  int n = nx + nu;
  int w = nx * odd_ld(n) + nx + wrapped_size(n) + wrapped_size(nu);
  return (w + 3) & ~3;
}
__host__ __device__ inline int blocks_per_instance(int lti, int N) { return lti ? 2 : N; }

// Per-instance solver state kept on the device between calls.
struct InstState {
  int iters;      // iterations run by the last solve
  int status;     // kConverged / kMaxIter / kNonFinite
  int momentum;   // iterations that read the previous iterate (momentum factor != 0)
  int pad;
  double c;       // last c^{i+1}
};

}  // namespace pimpc

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
// Tiled layout (one-thread-per-stage kernel of pimpc_solve_static): see admm_tps.cu.
// Halo-tile layout (tiled == 2, stage-varying instances, one thread per stage): see below.
// Blocked layout (tiled == 3, lanes owning 4-column blocks): see below.
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
constexpr int kFactorFailed = 4;
constexpr int kStalled = 5;
constexpr int kMaxNLtv = 32;
constexpr int kMaxNLti = 64;

struct Layout {
  int batch;
  int lti;
  int tiled;                       // 0: plain stage-major; 1: 32-stage tiles; 2: halo tiles;
                                   // 3: blocked stage-major
  const int *tw;                   // halo tiles: slots per tile (tiled == 2), else null
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
  int fine;              // the active list holds the fine items (one sub-chunk each)
  int bar_limit;         // polls of the grid barrier before it gives up (0: the default)
  int stale;             // entries of stopped instances still in the active list (marked -1)
  int pad[4];
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

// Halo tiles (tiled == 2). A tile has tw slots (tw <= 32); tile t holds stages t P - 1 .. t P + P
// in slots 0 .. tw - 1 (P = tw - 2): slots 1 .. P are the tile's own stages, slot 0 repeats the
// last own stage of tile t - 1 and slot tw - 1 the first own stage of tile t + 1, so that one
// iteration on a tile reads nothing outside it. Inside a tile every array is element-major:
// element e of slot s at e * tw + s (one thread per slot reads consecutive words). Stage data
// (per slot: G = [A | B] row-major nx x n, e, H packed lower row-major, M packed lower) occupies
// tile_block_words per tile, the iterates (z, v, theta, beta, lambda: 5 n elements per slot)
// tile_iter_words.
__host__ __device__ inline int halo_own(int tw) { return tw - 2; }
__host__ __device__ inline int halo_tiles(int N, int tw) { return (N + tw - 3) / (tw - 2); }
__host__ __device__ inline int packed_block_words(int nx, int nu) {
  const int n = nx + nu;
  return nx * n + nx + packed_size(n) + packed_size(nu);
}
__host__ __device__ inline int tile_block_words(int tw, int nx, int nu) {
  return (tw * packed_block_words(nx, nu) + 3) & ~3;
}
__host__ __device__ inline int tile_iter_words(int tw, int n) { return (tw * 5 * n + 3) & ~3; }
// Tile and slot of stage k's own copy.
__host__ __device__ inline void halo_slot(int tw, int k, int &t, int &s) {
  const int P = tw - 2;
  t = k / P;
  s = k - t * P + 1;
}
// The copies of stage k in neighbouring tiles: (tile, slot) pairs, returns how many (0..2).
__host__ __device__ inline int halo_copies(int tw, int N, int k, int *tt, int *ss) {
  int t, s, m = 0;
  halo_slot(tw, k, t, s);
  if (s == tw - 2 && t + 1 < halo_tiles(N, tw)) { tt[m] = t + 1; ss[m] = 0; ++m; }
  if (s == 1 && t >= 1) { tt[m] = t - 1; ss[m] = tw - 1; ++m; }
  return m;
}

// Blocked layout (tiled == 3). Stage-major like the plain layout, but built for lanes that own
// 4-column blocks (16-byte vector accesses in FP32):
//   [ G_k : nx rows of stride bl_ldg(n) ][ e_k : nx, padded to 4 ][ H_k as wrapped 4 x 4 block
//   diagonals ][ M_k as (scalar) wrapped diagonals, padded to 4 ]
// H_k (n x n, zero-padded to 4 nb, nb = ceil(n / 4)) is cut into 4 x 4 blocks S_{I,J}; for
// d = 0 .. nb/2 the block S_{I,(I+d) mod nb} is stored (blocks d and nb - d are transposes of
// each other, so this holds every block once). The diagonal blocks (d = 0) are symmetric: block
// I keeps its upper triangle, row by row (s00 s01 s02 s03 s11 s12 s13 s22 s23 s33), at 10 I,
// so a lane reads it as five 8-byte pairs (the region padded to 4 words). The other full block
// diagonals 1 <= d < Df = ceil(nb / 2) hold a block for every block row I: row a of block
// (d, I) sits at D0 + ((a (Df - 1) + d - 1) nb + I) * 4 (D0 = the padded diagonal region), so
// lanes reading row a of consecutive blocks read consecutive 16-byte words. For an even nb the
// middle diagonal d = nb/2 pairs block rows I and I + nb/2 (S_{I+nb/2,I} is the transpose of
// S_{I,I+nb/2}), so it is stored for I < nb/2 only, after the full ones: row a of its block I
// at D0 + 16 nb (Df - 1) + (a nb/2 + I) * 4. The G stride is chosen for
// the row products, where lane l of a group reads row l: FP32 rows are 4 nb words long when nb
// is odd (an odd number of 16-byte words: rows l = 0..7 start in distinct 16-byte bank groups)
// or 4 or 8 (lane l then reads, at step J, block (J + l) mod nb of its row, which again puts
// eight lanes on distinct bank groups: bl_rot), else 4 (nb + 1) words; FP64 rows are 4 nb + 2
// words. Iterates: [z | v | theta | beta | lambda], each padded to 4 (record
// 5 * bl_pad4(n)).
__host__ __device__ inline int bl_pad4(int m) { return (m + 3) & ~3; }
__host__ __device__ inline int bl_nb(int m) { return (m + 3) >> 2; }
__host__ __device__ inline int bl_diags(int nb) { return nb / 2 + 1; }
__host__ __device__ inline bool bl_pow2(int nb) { return (nb & (nb - 1)) == 0; }
// The row products read block (J + l) mod nb at step J on lane l.
__host__ __device__ inline bool bl_rot(int nb) { return nb == 4 || nb == 8; }
__host__ __device__ inline int bl_ldg(int n, int tsize) {
  const int nb = bl_nb(n);
  if (tsize != 4) return 4 * nb + 2;
  return ((nb & 1) || nb <= 2 || bl_rot(nb)) ? 4 * nb : 4 * (nb + 1);
}
// Block diagonals with a block for every block row (d = 0 included); an even nb adds the
// half-stored middle one.
__host__ __device__ inline int bl_full_diags(int nb) { return (nb + 1) >> 1; }
// Words of the diagonal blocks' upper triangles (10 per block, padded to 4).
__host__ __device__ inline int bl_diag_words(int nb) { return (10 * nb + 3) & ~3; }
// Slot of element (a, b), a <= b, in a diagonal block's upper triangle.
__host__ __device__ inline int bl_tri(int a, int b) { return a * 4 - ((a * (a - 1)) >> 1) + b - a; }
__host__ __device__ inline int bl_sym_words(int m) {
  const int nb = bl_nb(m);
  return bl_diag_words(nb) + 16 * nb * (bl_full_diags(nb) - 1) + ((nb & 1) ? 0 : 8 * nb);
}
// Whether element (a, b) of block (d, I) has a slot of its own (d <= nb/2; the middle diagonal
// of an even nb only for I < nb/2; a diagonal block only its upper triangle, a <= b).
__host__ __device__ inline bool bl_sym_stored(int nb, int d, int I, int a, int b) {
  if (d == 0) return a <= b;
  return d < bl_full_diags(nb) || I < (nb >> 1);
}
__host__ __device__ inline int bl_sym_index(int nb, int d, int I, int a, int b) {
  if (d == 0) return 10 * I + bl_tri(a, b);
  const int Df = bl_full_diags(nb), D0 = bl_diag_words(nb);
  if (d < Df) return D0 + ((a * (Df - 1) + d - 1) * nb + I) * 4 + b;
  return D0 + 16 * nb * (Df - 1) + (a * (nb >> 1) + I) * 4 + b;
}
// Offsets inside a blocked stage block: e, H, M; and the block size W.
__host__ __device__ inline int bl_oE(int nx, int nu, int tsize) { return nx * bl_ldg(nx + nu, tsize); }
__host__ __device__ inline int bl_oH(int nx, int nu, int tsize) { return bl_oE(nx, nu, tsize) + bl_pad4(nx); }
__host__ __device__ inline int bl_oM(int nx, int nu, int tsize) {
  return bl_oH(nx, nu, tsize) + bl_sym_words(nx + nu);
}
__host__ __device__ inline int bl_block_words(int nx, int nu, int tsize) {
  return bl_oM(nx, nu, tsize) + bl_pad4(wrapped_size(nu));
}
__host__ __device__ inline int bl_rec(int n) { return 5 * bl_pad4(n); }
// Lanes per stage of the blocked kernel (4 columns per lane).
__host__ __device__ inline int bl_group(int n) { return n <= 16 ? 4 : (n <= 32 ? 8 : 16); }

// Per-instance solver state kept on the device between calls.
struct InstState {
  int iters;      // iterations run by the last solve
  int status;     // kConverged / kMaxIter / kNonFinite
  int momentum;   // iterations that read the previous iterate (momentum factor != 0)
  int pad;
  double c;       // last c^{i+1}
};

}  // namespace pimpc

// affine.cu — score of the exact 3-way global alignment under affine gaps (sm_103a).
//
// The model is the sum-of-pairs score with natural gap costs: each pair's induced pairwise
// alignment (columns with a gap in both of its sequences deleted) scores sigma per residue pair,
// alpha per residue against a gap, and gamma once per maximal run of gaps in one sequence. The
// paper names affine gaps as future work (Sec. VI) without a definition; this is the reading the
// oracle implements.
//
// State of an alignment prefix: per pair, the kind of its last induced column (0 both residues or
// none, 1 gap in the pair's first sequence, 2 gap in its second). Only 13 of the 27 combinations
// can follow a column (the host-independent table below): the four moves with at least two
// residues set all three pairs, and each single-residue move sets two and keeps the third.
// Cell (i, j, k) holds one value per state; the kernel evaluates every (move, previous state)
// candidate in int32 with a -2^30 floor for states no prefix ends in. The moves and states are
// unrolled at compile time, so the state each candidate lands in and the gap runs it opens are
// constants, and a cell's 13 values live in registers.
//
// Layout and order. One CTA aligns one triplet at a time (a persistent queue, largest cube
// first). It sweeps the anti-diagonal planes d = i + j + k: the cells of a plane are independent,
// and their predecessors lie on planes d-1, d-2 and d-3, so four plane buffers rotate in the
// CTA's slice of global memory, indexed by (j, k) with 16 int32 per cell (13 used, four 16-byte
// loads per predecessor), one barrier per plane.
// This is the straightforward data-parallel form, not the register-tiled engine of the linear
// model: it serves the affine model at moderate sizes (the 4,096-triplet batch runs ~10 planes
// of 13-state cells per CTA at a time).
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

namespace trioseq {

namespace {

constexpr int kAffNeg = -(1 << 30);  // a state no prefix ends in
constexpr int kAffStates = kAffineStates;
constexpr int kAffStride = 16;       // int32 per cell in the plane buffers (13 used, 64 bytes)
constexpr int kAffThreads = 256;

// The 13 reachable states as kinds (pair 01, pair 02, pair 12); 0 both residues or none, 1 gap
// in the pair's first sequence, 2 gap in its second. Compile-time, so that with the loops over
// moves and states unrolled every state index and opening count folds to a constant and the 13
// values of a cell stay in registers.
__host__ __device__ constexpr int st_kind(int s, int pq) {
  constexpr int8_t t[kAffineStates][3] = {
      {0, 0, 0}, {0, 2, 2}, {2, 0, 1}, {1, 1, 0}, {2, 2, 0}, {2, 2, 1}, {2, 2, 2},
      {1, 0, 2}, {1, 1, 2}, {1, 2, 2}, {0, 1, 1}, {1, 1, 1}, {2, 1, 1}};
  return t[s][pq];
}

__host__ __device__ constexpr int st_index(int k01, int k02, int k12) {
  for (int s = 0; s < kAffineStates; ++s)
    if (st_kind(s, 0) == k01 && st_kind(s, 1) == k02 && st_kind(s, 2) == k12) return s;
  return 0;  // unreachable combinations never occur
}

// moves in Eq. 1's listing order: 111 110 101 011 100 010 001
__host__ __device__ constexpr int mv(int m, int q) {
  constexpr int8_t t[7][3] = {{1, 1, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
                              {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  return t[m][q];
}

// kind a move gives the pair (p0, p1): 0 untouched (gap in both), 1 both residues, 2 gap in p0,
// 3 gap in p1
__host__ __device__ constexpr int move_kind(int m, int pq) {
  const int p0 = pq == 2 ? 1 : 0, p1 = pq == 0 ? 1 : 2;
  const int r0 = mv(m, p0), r1 = mv(m, p1);
  return (!r0 && !r1) ? 0 : ((r0 && r1) ? 1 : (r0 ? 3 : 2));
}

// new state and number of gap runs opened when move m follows state s
__host__ __device__ constexpr int next_state(int m, int s) {
  int k[3] = {0, 0, 0};
  for (int pq = 0; pq < 3; ++pq) {
    const int mk = move_kind(m, pq);
    k[pq] = mk == 0 ? st_kind(s, pq) : (mk == 1 ? 0 : mk - 1);
  }
  return st_index(k[0], k[1], k[2]);
}
__host__ __device__ constexpr int opens(int m, int s) {
  int n = 0;
  for (int pq = 0; pq < 3; ++pq) {
    const int mk = move_kind(m, pq);
    if (mk >= 2 && st_kind(s, pq) != mk - 1) ++n;
  }
  return n;
}

}  // namespace

__global__ void __launch_bounds__(kAffThreads) affine_kernel(const AffineParams p) {
  __shared__ int sig[kMaxAlphabet * kMaxAlphabet];
  __shared__ int next;
  const int KP = p.KP;
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) sig[e] = p.sub[e];
  int32_t* const base = p.planes + (int64_t)blockIdx.x * 4 * p.plane_cells * kAffStride;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next = atomicAdd(p.queue, 1);
    __syncthreads();
    const int q = next;
    if (q >= p.n) return;
    const TripDesc& d = p.desc[p.tasks[q].trip];
    const int a = d.len[0], b = d.len[1], c = d.len[2];
    const int8_t* S0 = p.seq + d.s_off[0];
    const int8_t* S1 = p.seq + d.s_off[1];
    const int8_t* S2 = p.seq + d.s_off[2];
    const int C = c + 1;
    const int gap = p.gap, go = p.gap_open;
    // plane d lives in buffer d & 3; cell (j, k) at (j * C + k) * 16
    for (int dd = 0; dd <= a + b + c; ++dd) {
      int32_t* cur = base + (int64_t)(dd & 3) * p.plane_cells * kAffStride;
      const int jlo = max(0, dd - a - c), jhi = min(b, dd);
      const int64_t rows = jhi - jlo + 1;
      for (int64_t e = threadIdx.x; e < rows * C; e += blockDim.x) {
        const int j = jlo + (int)(e / C), k = (int)(e % C);
        const int i = dd - j - k;
        if (i < 0 || i > a) continue;
        int F[kAffStates];
#pragma unroll
        for (int s = 0; s < kAffStates; ++s) F[s] = kAffNeg;
        if (dd == 0) F[0] = 0;
        const int x = i > 0 ? (int)S0[i - 1] : 0, y = j > 0 ? (int)S1[j - 1] : 0,
                  z = k > 0 ? (int)S2[k - 1] : 0;
#pragma unroll
        for (int m = 0; m < 7; ++m) {
          const int di = mv(m, 0), dj = mv(m, 1), dk = mv(m, 2);
          if (dd == 0 || i < di || j < dj || k < dk) continue;
          const int4* G = reinterpret_cast<const int4*>(
              base + (int64_t)((dd - di - dj - dk) & 3) * p.plane_cells * kAffStride +
              ((int64_t)(j - dj) * C + (k - dk)) * kAffStride);
          const int4 g0 = G[0], g1 = G[1], g2 = G[2], g3 = G[3];
          const int g[16] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w,
                             g2.x, g2.y, g2.z, g2.w, g3.x, g3.y, g3.z, g3.w};
          // the column's pair scores: sigma per residue pair, alpha per residue against a gap
          int fixed = 0;
          fixed += move_kind(m, 0) == 1 ? sig[x * KP + y] : (move_kind(m, 0) ? gap : 0);
          fixed += move_kind(m, 1) == 1 ? sig[x * KP + z] : (move_kind(m, 1) ? gap : 0);
          fixed += move_kind(m, 2) == 1 ? sig[y * KP + z] : (move_kind(m, 2) ? gap : 0);
#pragma unroll
          for (int s = 0; s < kAffStates; ++s) {
            const int ns = next_state(m, s);
            F[ns] = max(F[ns], g[s] + fixed + opens(m, s) * go);
          }
        }
        int4* out = reinterpret_cast<int4*>(cur + ((int64_t)j * C + k) * kAffStride);
        // a state no prefix ends in stays at the floor instead of drifting below it
        int v[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = s < kAffStates ? max(F[s], kAffNeg) : kAffNeg;
        out[0] = make_int4(v[0], v[1], v[2], v[3]);
        out[1] = make_int4(v[4], v[5], v[6], v[7]);
        out[2] = make_int4(v[8], v[9], v[10], v[11]);
        out[3] = make_int4(v[12], v[13], v[14], v[15]);
        if (i == a && j == b && k == c) {
          int best = F[0];
#pragma unroll
          for (int s = 1; s < kAffStates; ++s) best = max(best, F[s]);
          p.scores[d.out_idx] = best;
        }
      }
      __syncthreads();
    }
  }
}

int affine_threads() { return kAffThreads; }

int affine_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, affine_kernel, kAffThreads,
                                                       0) == cudaSuccess
             ? 0
             : -2;
}

int launch_affine(const AffineParams& p, int grid, void* stream) {
  affine_kernel<<<grid, kAffThreads, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trioseq

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
// candidate in int32 with a -2^30 floor for states no prefix ends in.
//
// Layout and order. One CTA aligns one triplet at a time (a persistent queue, largest cube
// first). It sweeps the anti-diagonal planes d = i + j + k: the cells of a plane are independent,
// and their predecessors lie on planes d-1, d-2 and d-3, so four plane buffers rotate in the
// CTA's slice of global memory, indexed by (j, k) with 13 int32 per cell, one barrier per plane.
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
constexpr int kAffThreads = 256;

// The 13 reachable states as (kind of pair 01, pair 02, pair 12).
__constant__ int8_t c_state_kind[kAffStates][3] = {
    {0, 0, 0}, {0, 2, 2}, {2, 0, 1}, {1, 1, 0}, {2, 2, 0}, {2, 2, 1}, {2, 2, 2},
    {1, 0, 2}, {1, 1, 2}, {1, 2, 2}, {0, 1, 1}, {1, 1, 1}, {2, 1, 1}};

__constant__ int c_pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};

__device__ __forceinline__ int state_of(int k01, int k02, int k12) {
  // inverse of c_state_kind (unreachable combinations never occur)
  const int key = k01 * 9 + k02 * 3 + k12;
  switch (key) {
    case 0: return 0;
    case 8: return 1;
    case 19: return 2;
    case 12: return 3;
    case 24: return 4;
    case 25: return 5;
    case 26: return 6;
    case 11: return 7;
    case 14: return 8;
    case 17: return 9;
    case 4: return 10;
    case 13: return 11;
    case 22: return 12;
  }
  return 0;
}

}  // namespace

__global__ void __launch_bounds__(kAffThreads) affine_kernel(const AffineParams p) {
  __shared__ int sig[kMaxAlphabet * kMaxAlphabet];
  __shared__ int next;
  const int KP = p.KP;
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) sig[e] = p.sub[e];
  int32_t* const base = p.planes + (int64_t)blockIdx.x * 4 * p.plane_cells * kAffStates;
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
    // plane d lives in buffer d & 3; cell (j, k) at ((j * C + k) * 13)
    for (int dd = 0; dd <= a + b + c; ++dd) {
      int32_t* cur = base + (int64_t)(dd & 3) * p.plane_cells * kAffStates;
      const int jlo = max(0, dd - a - c), jhi = min(b, dd);
      const int64_t rows = jhi - jlo + 1;
      for (int64_t e = threadIdx.x; e < rows * C; e += blockDim.x) {
        const int j = jlo + (int)(e / C), k = (int)(e % C);
        const int i = dd - j - k;
        if (i < 0 || i > a) continue;
        int F[kAffStates];
#pragma unroll
        for (int s = 0; s < kAffStates; ++s) F[s] = kAffNeg;
        if (dd == 0) {
          F[0] = 0;
        } else {
          for (int m = 0; m < 7; ++m) {
            // moves in Eq. 1's listing order: 111 110 101 011 100 010 001
            const int di = (m == 0 || m == 1 || m == 2 || m == 4);
            const int dj = (m == 0 || m == 1 || m == 3 || m == 5);
            const int dk = (m == 0 || m == 2 || m == 3 || m == 6);
            if (i < di || j < dj || k < dk) continue;
            const int pd = dd - di - dj - dk;
            const int32_t* G = base + (int64_t)(pd & 3) * p.plane_cells * kAffStates +
                               ((int64_t)(j - dj) * C + (k - dk)) * kAffStates;
            const int r[3] = {di ? (int)S0[i - 1] : -1, dj ? (int)S1[j - 1] : -1,
                              dk ? (int)S2[k - 1] : -1};
            // per pair: 0 untouched (both gaps), 1 both residues, 2 gap in first, 3 gap in second
            int kind[3], fixed = 0;
#pragma unroll
            for (int pq = 0; pq < 3; ++pq) {
              const int x = r[c_pairs[pq][0]], y = r[c_pairs[pq][1]];
              if (x < 0 && y < 0) {
                kind[pq] = 0;
              } else if (x >= 0 && y >= 0) {
                kind[pq] = 1;
                fixed += sig[x * KP + y];
              } else {
                kind[pq] = x < 0 ? 2 : 3;
                fixed += p.gap;
              }
            }
            for (int s = 0; s < kAffStates; ++s) {
              const int g = G[s];
              if (g <= kAffNeg / 2) continue;
              int cand = g + fixed, nk[3];
#pragma unroll
              for (int pq = 0; pq < 3; ++pq) {
                const int prev = c_state_kind[s][pq];
                if (kind[pq] == 0) {
                  nk[pq] = prev;
                } else if (kind[pq] == 1) {
                  nk[pq] = 0;
                } else {
                  const int want = kind[pq] - 1;  // 1: gap in first, 2: gap in second
                  if (prev != want) cand += p.gap_open;
                  nk[pq] = want;
                }
              }
              const int ns = state_of(nk[0], nk[1], nk[2]);
              F[ns] = max(F[ns], cand);
            }
          }
        }
        int32_t* out = cur + ((int64_t)j * C + k) * kAffStates;
#pragma unroll
        for (int s = 0; s < kAffStates; ++s) out[s] = F[s];
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

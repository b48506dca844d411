// kernels.cu — sm_103a kernels of the 3-way alignment engine.
//
// wavefront_kernel<NJ, NK, TB>: persistent "column task" engine for Eq. 1.
//   The (j,k) plane of each triplet is cut into column blocks of WJ x WK cells
//   (WJ = 4*NJ, WK = 8*NK). One warp owns one block at a time and sweeps the whole i axis
//   through it: lane (r, lc) of the 4 x 8 lane grid holds an NJ x NK register tile of the
//   current i-slice and works on slice s = t - r - lc at step t, so each lane's j- and k-halo
//   for slice s was produced by its upper / left neighbour lane one step earlier and arrives by
//   warp shuffle (the anti-diagonal skew of the paper's warp kernel, Sec. IV-B, rebuilt for
//   int32 on one warp per column block).
//   Column blocks exchange their boundary faces through global memory (L2): block (J,K) reads
//   the j-face written by (J-1,K) and the k-face written by (J,K-1), one int32 per face cell per
//   slice. A producer publishes how many steps it has completed every TI steps with a release
//   store; a consumer waits (bounded, acquire) before it touches a face row. Tasks are handed
//   out through one atomic queue in an order where every producer precedes its consumers, so
//   the engine cannot deadlock even when not all warps are resident.
//   TB = true additionally keeps traceback keys (8*M' + 7, see engine.h) and streams one 4-bit
//   code per cell to HBM (rank of the winning move, 8 cells per 32-bit word, one 32-byte record
//   per lane per step).
//
// walk_kernel: follows the stored codes from (a,b,c) back to the origin for each traceback
//   request and writes the three aligned rows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

namespace trioseq {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Lane-0 wait until *flag >= need. `cached` keeps the last value seen. Gives up (returns false)
// when the flag has not moved for wait_ns nanoseconds.
__device__ __noinline__ bool wait_flag(const int* flag, int need, int* cached, int64_t wait_ns) {
  int last = *cached;
  if (last >= need) return true;
  uint64_t t0 = global_ns();
  for (;;) {
    const int v = ld_acquire(flag);
    if (v >= need) {
      *cached = v;
      return true;
    }
    const uint64_t now = global_ns();
    if (v != last) {
      last = v;
      t0 = now;
    } else if ((int64_t)(now - t0) > wait_ns) {
      *cached = v;
      return false;
    }
    __nanosleep(128);
  }
}

constexpr unsigned kFull = 0xffffffffu;

}  // namespace

// Resident CTAs per SM the register budget is sized for (4 warps each).
template <int NJ, int NK>
struct MinBlocks {
  static constexpr int value = (NJ * NK >= 64) ? 2 : ((NJ * NK >= 32) ? 3 : 4);
};

template <int NJ, int NK, bool TB>
__global__ void __launch_bounds__(kWarpsPerCta * 32, MinBlocks<NJ, NK>::value)
    wavefront_kernel(const WaveParams p) {
  static_assert(NJ % 4 == 0 && NK % 4 == 0, "tile sides must be multiples of 4");
  constexpr int WJ = kPR * NJ, WK = kPC * NK;
  constexpr int PJ = WJ + 4, PK = WK + 4;  // padded profile rows spread lanes over banks
  constexpr int W = NJ * NK / 8;           // code words per lane per step
  extern __shared__ int4 smem4[];
  int* smem = reinterpret_cast<int*>(smem4);
  const int KP = p.KP;
  const int VIRT = KP - 1;
  const int sigN = (KP * KP + 3) & ~3;
  int* sig = smem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* profJ = smem + sigN + warp * (KP * (PJ + PK));
  int* profK = profJ + KP * PJ;
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) sig[e] = p.sig[e];
  __syncthreads();
  const int r = lane >> 3, lc = lane & 7;

  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(p.queue, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= p.ntasks) return;
    const Task tk = p.tasks[task];
    const TripDesc& d = p.desc[tk.trip];
    const int a = d.len[0], b = d.len[1], c = d.len[2];
    const int nJ = d.nJ, nK = d.nK, T = d.T;
    const int J = tk.J, K = tk.K;
    const int8_t* S0 = p.seq + d.s_off[0];
    const int8_t* S1 = p.seq + d.s_off[1];
    const int8_t* S2 = p.seq + d.s_off[2];
    const int j0 = J * WJ + r * NJ, k0 = K * WK + lc * NK;

    // Substitution profiles of this block: profJ[x][jl] = sigma''(x, y_(J*WJ+jl)),
    // profK[x][kl] = sigma''(x, z_(K*WK+kl)); residue index 0 and beyond the end are VIRT.
    __syncwarp();
    for (int e = lane; e < KP * WJ; e += 32) {
      const int x = e / WJ, jl = e - x * WJ, j = J * WJ + jl;
      const int y = (j >= 1 && j <= b) ? (int)S1[j - 1] : VIRT;
      profJ[x * PJ + jl] = sig[x * KP + y];
    }
    for (int e = lane; e < KP * WK; e += 32) {
      const int x = e / WK, kl = e - x * WK, k = K * WK + kl;
      const int z = (k >= 1 && k <= c) ? (int)S2[k - 1] : VIRT;
      profK[x * PK + kl] = sig[x * KP + z];
    }
    // sigma''(y_j, z_k) is the same for every i: keep this lane's tile of it in registers.
    int Cv[NJ][NK];
    {
      int yo[NJ], zv[NK];
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp) {
        const int j = j0 + pp;
        yo[pp] = ((j >= 1 && j <= b) ? (int)S1[j - 1] : VIRT) * KP;
      }
#pragma unroll
      for (int qq = 0; qq < NK; ++qq) {
        const int k = k0 + qq;
        zv[qq] = (k >= 1 && k <= c) ? (int)S2[k - 1] : VIRT;
      }
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
        for (int qq = 0; qq < NK; ++qq) Cv[pp][qq] = sig[yo[pp] + zv[qq]];
    }
    __syncwarp();

    // Owner of the final cell (a, b, c).
    const bool owns_end = (J == b / WJ) && (K == c / WK) && (r == (b % WJ) / NJ) &&
                          (lc == (c % WK) / NK);
    const int end_p = b % NJ, end_q = c % NK;

    int P[NJ][NK];
    int rowPrev[NK + 1], colPrev[NJ], rowCur[NK + 1], colCur[NJ], nxtRow[NK + 1], nxtCol[NJ];
#pragma unroll
    for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
      for (int qq = 0; qq < NK; ++qq) P[pp][qq] = kNeg;
      colPrev[pp] = kNeg;
      colCur[pp] = kNeg;
      nxtCol[pp] = kNeg;
    }
#pragma unroll
    for (int qq = 0; qq <= NK; ++qq) {
      rowPrev[qq] = kNeg;
      rowCur[qq] = kNeg;
      nxtRow[qq] = kNeg;
    }
    // M'[-1][-1][-1] = 0 feeds the origin through the (1,1,1) move (stored as 8*0+7 with keys).
    if (J == 0 && K == 0 && lane == 0) rowPrev[0] = TB ? 7 : 0;

    const int64_t planeJ = (int64_t)(a + 1) * d.rowJ;
    const int64_t planeK = (int64_t)(a + 1) * d.rowK;
    const int* fj_in = p.faces + d.fj_off + (int64_t)(J - 1) * planeJ;
    int* fj_out = p.faces + d.fj_off + (int64_t)J * planeJ;
    const int* fk_in = p.faces + d.fk_off + (int64_t)(K - 1) * planeK;
    int* fk_out = p.faces + d.fk_off + (int64_t)K * planeK;
    const bool has_fj_out = (J + 1 < nJ), has_fk_out = (K + 1 < nK);
    const int* progJ = p.progress + d.prog_base + (int64_t)(J - 1) * nK + K;
    const int* progK = p.progress + d.prog_base + (int64_t)J * nK + (K - 1);
    int* progMe = p.progress + d.prog_base + (int64_t)J * nK + K;
    int cachedJ = 0, cachedK = 0;
    uint32_t* code_base =
        TB ? p.codes + d.code_off + (int64_t)(J * nK + K) * T * 32 * W + lane * W : nullptr;

    bool ok = true;
    // Fetch the face halos of the edge lanes for step tt into nxtRow / nxtCol. The face row a
    // lane reads was written by the producer lane at producer step tt + kPR - 1 (j-face) or
    // tt + kPC - 1 (k-face); lane 0 first waits until the producer has published those steps.
#define TRIOSEQ_LOAD_EDGES(tt)                                                                  \
  {                                                                                             \
    bool okl = true;                                                                            \
    if (lane == 0) {                                                                            \
      if (J > 0) okl = wait_flag(progJ, min((tt) + kPR, T), &cachedJ, p.wait_ns);               \
      if (okl && K > 0) okl = wait_flag(progK, min((tt) + kPC, T), &cachedK, p.wait_ns);        \
    }                                                                                           \
    ok = __shfl_sync(kFull, okl, 0);                                                            \
    __syncwarp();                                                                               \
    const int ss = (tt) - r - lc;                                                               \
    const bool sv = ok && ss >= 0 && ss <= a;                                                   \
    if (r == 0) {                                                                               \
      if (J > 0 && sv) {                                                                        \
        const int* src = fj_in + (int64_t)ss * d.rowJ + k0 + 4;                                 \
        nxtRow[0] = (K == 0 && lc == 0) ? kNeg : __ldcg(src - 1);                               \
        _Pragma("unroll") for (int q4 = 0; q4 < NK / 4; ++q4) {                                 \
          const int4 v = __ldcg(reinterpret_cast<const int4*>(src) + q4);                       \
          nxtRow[1 + 4 * q4] = v.x;                                                             \
          nxtRow[2 + 4 * q4] = v.y;                                                             \
          nxtRow[3 + 4 * q4] = v.z;                                                             \
          nxtRow[4 + 4 * q4] = v.w;                                                             \
        }                                                                                       \
      } else {                                                                                  \
        _Pragma("unroll") for (int qq = 0; qq <= NK; ++qq) nxtRow[qq] = kNeg;                   \
      }                                                                                         \
    }                                                                                           \
    if (lc == 0) {                                                                              \
      if (K > 0 && sv) {                                                                        \
        const int* src = fk_in + (int64_t)ss * d.rowK + j0 + 4;                                 \
        _Pragma("unroll") for (int p4 = 0; p4 < NJ / 4; ++p4) {                                 \
          const int4 v = __ldcg(reinterpret_cast<const int4*>(src) + p4);                       \
          nxtCol[4 * p4] = v.x;                                                                 \
          nxtCol[4 * p4 + 1] = v.y;                                                             \
          nxtCol[4 * p4 + 2] = v.z;                                                             \
          nxtCol[4 * p4 + 3] = v.w;                                                             \
        }                                                                                       \
      } else {                                                                                  \
        _Pragma("unroll") for (int pp = 0; pp < NJ; ++pp) nxtCol[pp] = kNeg;                    \
      }                                                                                         \
    }                                                                                           \
  }

    TRIOSEQ_LOAD_EDGES(0);
    for (int t = 0; ok && t < T; ++t) {
      const int s = t - r - lc;
      if (r == 0) {
#pragma unroll
        for (int qq = 0; qq <= NK; ++qq) rowCur[qq] = nxtRow[qq];
      }
      if (lc == 0) {
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) colCur[pp] = nxtCol[pp];
      }
      if (t + 1 < T) TRIOSEQ_LOAD_EDGES(t + 1);
      if (!ok) break;

      if (s >= 0 && s <= a) {
        const int x = (s == 0) ? VIRT : (int)__ldg(S0 + s - 1);
        int A[NJ], B[NK];
        {
          const int4* pa = reinterpret_cast<const int4*>(profJ + x * PJ + r * NJ);
#pragma unroll
          for (int p4 = 0; p4 < NJ / 4; ++p4) {
            const int4 v = pa[p4];
            A[4 * p4] = v.x;
            A[4 * p4 + 1] = v.y;
            A[4 * p4 + 2] = v.z;
            A[4 * p4 + 3] = v.w;
          }
          const int4* pb = reinterpret_cast<const int4*>(profK + x * PK + lc * NK);
#pragma unroll
          for (int q4 = 0; q4 < NK / 4; ++q4) {
            const int4 v = pb[q4];
            B[4 * q4] = v.x;
            B[4 * q4 + 1] = v.y;
            B[4 * q4 + 2] = v.z;
            B[4 * q4 + 3] = v.w;
          }
        }
        int Q[NJ][NK];
        uint32_t cw[W > 0 ? W : 1];
#pragma unroll
        for (int w = 0; w < (W > 0 ? W : 1); ++w) cw[w] = 0u;
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
          for (int qq = 0; qq < NK; ++qq) {
            // Predecessors of cell (s, j0+pp, k0+qq): previous slice (P, prev halos) and this
            // slice (Q, current halos).
            const int Pd = (pp == 0) ? rowPrev[qq] : (qq == 0 ? colPrev[pp - 1] : P[pp - 1][qq - 1]);
            const int Pxy = (pp == 0) ? rowPrev[qq + 1] : P[pp - 1][qq];
            const int Pxz = (qq == 0) ? colPrev[pp] : P[pp][qq - 1];
            const int Sx = P[pp][qq];
            const int Myz = (pp == 0) ? rowCur[qq] : (qq == 0 ? colCur[pp - 1] : Q[pp - 1][qq - 1]);
            const int Sy = (pp == 0) ? rowCur[qq + 1] : Q[pp - 1][qq];
            const int Sz = (qq == 0) ? colCur[pp] : Q[pp][qq - 1];
            if (!TB) {
              // max{ Pd+A+B+C, Pxy+A, Pxz+B, Myz+C, Sx, Sy, Sz } (shifted frame, engine.h)
              const int d0 = Pd + A[pp] + B[qq];
              int u = max(Pxy + A[pp], Sx);
              u = max(Pxz + B[qq], u);
              const int w = max(d0, Myz);
              int v = max(w + Cv[pp][qq], u);
              Q[pp][qq] = max(v, max(Sy, Sz));
            } else {
              // Keys: rank offsets 0,-1,-2,-3,-4,-5,-6 for moves 111,110,101,011,100,010,001.
              const int d0 = Pd + A[pp] + B[qq];
              const int w = max(d0, Myz - 3);
              int u = max(Pxy + (A[pp] - 1), Sx - 4);
              u = max(Pxz + (B[qq] - 2), u);
              int v = max(w + Cv[pp][qq], u);
              v = max(v, max(Sy - 5, Sz - 6));
              const int n = pp * NK + qq;
              cw[n >> 3] |= (uint32_t)(v & 7) << (4 * (n & 7));
              Q[pp][qq] = v | 7;
            }
          }
        }
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
          for (int qq = 0; qq < NK; ++qq) P[pp][qq] = Q[pp][qq];

        if (TB) {
          uint32_t* dst = code_base + (int64_t)t * 32 * W;
          if (W % 4 == 0) {
#pragma unroll
            for (int w4 = 0; w4 < W / 4; ++w4)
              reinterpret_cast<uint4*>(dst)[w4] =
                  make_uint4(cw[4 * w4], cw[4 * w4 + 1], cw[4 * w4 + 2], cw[4 * w4 + 3]);
          } else {
#pragma unroll
            for (int w2 = 0; w2 < W / 2; ++w2)
              reinterpret_cast<uint2*>(dst)[w2] = make_uint2(cw[2 * w2], cw[2 * w2 + 1]);
          }
        }
        if (r == kPR - 1 && has_fj_out) {
          int4* dst = reinterpret_cast<int4*>(fj_out + (int64_t)s * d.rowJ + k0 + 4);
#pragma unroll
          for (int q4 = 0; q4 < NK / 4; ++q4)
            dst[q4] = make_int4(P[NJ - 1][4 * q4], P[NJ - 1][4 * q4 + 1], P[NJ - 1][4 * q4 + 2],
                                P[NJ - 1][4 * q4 + 3]);
        }
        if (lc == kPC - 1 && has_fk_out) {
          int4* dst = reinterpret_cast<int4*>(fk_out + (int64_t)s * d.rowK + j0 + 4);
#pragma unroll
          for (int p4 = 0; p4 < NJ / 4; ++p4)
            dst[p4] = make_int4(P[4 * p4][NK - 1], P[4 * p4 + 1][NK - 1], P[4 * p4 + 2][NK - 1],
                                P[4 * p4 + 3][NK - 1]);
        }
        if (owns_end && s == a) {
          int v = 0;
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int qq = 0; qq < NK; ++qq)
              if (pp == end_p && qq == end_q) v = P[pp][qq];
          p.scores[d.out_idx] = (TB ? (v >> 3) : v) + d.score_base;
        }
      }

      // Hand this slice's boundary to the lanes below (j) and to the right (k).
      {
        int sendRow[NK + 1], sendCol[NJ];
        sendRow[0] = colCur[NJ - 1];
#pragma unroll
        for (int qq = 0; qq < NK; ++qq) sendRow[qq + 1] = P[NJ - 1][qq];
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) sendCol[pp] = P[pp][NK - 1];
#pragma unroll
        for (int qq = 0; qq <= NK; ++qq) {
          const int v = __shfl_up_sync(kFull, sendRow[qq], kPC);
          rowPrev[qq] = rowCur[qq];
          if (r > 0) rowCur[qq] = v;
        }
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
          const int v = __shfl_up_sync(kFull, sendCol[pp], 1);
          colPrev[pp] = colCur[pp];
          if (lc > 0) colCur[pp] = v;
        }
      }
      if ((t + 1) % p.TI == 0 || t + 1 == T) {
        __syncwarp();
        if (lane == 0) st_release(progMe, t + 1);
      }
    }
#undef TRIOSEQ_LOAD_EDGES
    if (!ok) {
      if (lane == 0) atomicOr(p.err, 1);
      return;
    }
  }
}

__global__ void walk_kernel(const WalkParams p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.ntb) return;
  const TripDesc& d = p.desc[p.tb_trips[q]];
  const int a = d.len[0], b = d.len[1], c = d.len[2];
  const int NJ = p.NJ, NK = p.NK, WJ = kPR * NJ, WK = kPC * NK, W = NJ * NK / 8;
  const int8_t* S0 = p.seq + d.s_off[0];
  const int8_t* S1 = p.seq + d.s_off[1];
  const int8_t* S2 = p.seq + d.s_off[2];
  const int cap = p.row_cap[q];
  uint8_t* row0 = p.rows + p.row_off[q];
  uint8_t* row1 = row0 + cap;
  uint8_t* row2 = row1 + cap;
  const uint32_t* codes = p.codes + d.code_off;
  int i = a, j = b, k = c, n = 0;
  while (i > 0 || j > 0 || k > 0) {
    const int J = j / WJ, K = k / WK;
    const int jl = j - J * WJ, kl = k - K * WK;
    const int rr = jl / NJ, cc = kl / NK;
    const int t = i + rr + cc, ln = rr * kPC + cc;
    const int e = (jl - rr * NJ) * NK + (kl - cc * NK);
    const uint32_t word =
        __ldg(codes + ((((int64_t)(J * d.nK + K) * d.T + t) * 32 + ln) * W + (e >> 3)));
    const int rank = (word >> (4 * (e & 7))) & 7;
    // rank -> move (Eq. 1 listing order, rank 7 first)
    const int di = (rank == 7 || rank == 6 || rank == 5 || rank == 3) ? 1 : 0;
    const int dj = (rank == 7 || rank == 6 || rank == 4 || rank == 2) ? 1 : 0;
    const int dk = (rank == 7 || rank == 5 || rank == 4 || rank == 1) ? 1 : 0;
    if (rank == 0 || n >= cap || i < di || j < dj || k < dk) {
      atomicOr(p.err, 2);
      p.aln_len[q] = -1;
      return;
    }
    const int pos = cap - 1 - n;
    row0[pos] = di ? (uint8_t)S0[i - 1] : (uint8_t)255;
    row1[pos] = dj ? (uint8_t)S1[j - 1] : (uint8_t)255;
    row2[pos] = dk ? (uint8_t)S2[k - 1] : (uint8_t)255;
    i -= di;
    j -= dj;
    k -= dk;
    ++n;
  }
  p.aln_len[q] = n;
}

namespace {

template <int NJ, int NK, bool TB>
const void* kptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, TB>);
}

const void* pick(int nj, int nk, bool tb) {
  if (nj == 8 && nk == 8) return tb ? kptr<8, 8, true>() : kptr<8, 8, false>();
  if (nj == 4 && nk == 8) return tb ? kptr<4, 8, true>() : kptr<4, 8, false>();
  if (nj == 4 && nk == 4) return tb ? kptr<4, 4, true>() : kptr<4, 4, false>();
  return nullptr;
}

}  // namespace

size_t wavefront_smem_bytes(int nj, int nk, int KP) {
  const int WJ = kPR * nj, WK = kPC * nk;
  const size_t sigN = (size_t)((KP * KP + 3) & ~3);
  return (sigN + (size_t)kWarpsPerCta * KP * ((WJ + 4) + (WK + 4))) * sizeof(int);
}

int wavefront_occupancy(int nj, int nk, bool tb, size_t smem, int* blocks_per_sm) {
  const void* k = pick(nj, nk, tb);
  if (!k) return -1;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return -2;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kWarpsPerCta * 32, smem) !=
      cudaSuccess)
    return -2;
  return 0;
}

int launch_wavefront(int nj, int nk, bool tb, const WaveParams& p, int grid, size_t smem,
                     void* stream) {
  const void* k = pick(nj, nk, tb);
  if (!k) return -1;
  void* args[] = {const_cast<WaveParams*>(&p)};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kWarpsPerCta * 32), args, smem,
                                         (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : -2;
}

int launch_walk(const WalkParams& p, void* stream) {
  if (p.ntb <= 0) return 0;
  const int bs = 64;
  walk_kernel<<<(p.ntb + bs - 1) / bs, bs, 0, (cudaStream_t)stream>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trioseq

// wavefront.cuh — the persistent wavefront kernel of the 3-way alignment engine (sm_103a).
//
// wavefront_kernel<NJ, NK, TB>: persistent "column task" engine for Eq. 1.
//   The (j,k) plane of each triplet is cut into column blocks of WJ x WK cells
//   (WJ = 4*NJ, WK = 8*NK). One warp owns one block at a time and sweeps the whole i axis
//   through it: lane (r, lc) of the 4 x 8 lane grid holds an NJ x NK register tile of the
//   current i-slice and works on slice s = t - r - lc at step t, so each lane's j- and k-halo
//   for slice s was produced by its upper / left neighbour lane one step earlier and arrives by
//   warp shuffle (the anti-diagonal skew of the paper's warp kernel, Sec. IV-B, rebuilt for
//   int32 on one warp per column block).
//   Column blocks exchange boundary records through global memory (L2): block (J,K) reads the
//   j-records written by (J-1,K) and the k-records written by (J,K-1) (engine.h). A producer
//   publishes how many steps it has completed every TI steps with a release store. The
//   consumer's edge lanes need the records of step t; every lane loads one 16-byte piece of
//   them from L2 one or two steps early (after lane 0 has acquired the producer's progress,
//   bounded wait) and parks it in a small per-warp shared-memory ring. All lanes then read
//   their halo from the ring and select it against the shuffled value; loads and stores that
//   only some lanes make are predicated, so the step loop has no lane-divergent branches.
//   Tasks come from one atomic queue in an order where every producer precedes its consumers,
//   so the engine cannot deadlock even when not all warps are resident.
//   TB = true additionally keeps traceback keys (8*M' + 7, engine.h) and streams one 4-bit code
//   per cell to HBM (one record of NJ*NK/8 words per lane per step).
//
//
// Included by kernels.cu (global alignment, both modes) and kernels_variants.cu (semi-global
// and local, score mode), so the instantiations compile as separate translation units.
#pragma once
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

// Lane-0 wait until *flag >= need. `cached` keeps the last value seen. Polls with acquire loads
// (the satisfying one orders the record loads that follow; unlike a fence it does not wait for
// this warp's own record stores in flight) and exponential back-off up to 256 ns, light on L2
// while many warps wait and at most a fraction of a step late. Gives up (returns false) when
// the flag has not moved for wait_ns. Inlined: an out-of-line call in the step loop, even one
// never taken, cost a lone warp 6-8% of its step (the call's register save/restore constrains the
// whole loop body), and the main-line kernel 5%.
__device__ __forceinline__ bool wait_flag(const int* flag, int need, int* cached, int64_t wait_ns) {
  int v = ld_acquire(flag);
  if (v >= need) {
    *cached = v;
    return true;
  }
  int last = v;
  unsigned ns = 32;
  uint64_t t0 = global_ns();
  for (;;) {
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
    v = ld_acquire(flag);
    if (v >= need) {
      *cached = v;
      return true;
    }
    const uint64_t now = global_ns();
    if (v != last) {
      last = v;
      t0 = now;
      ns = 32;
    } else if ((int64_t)(now - t0) > wait_ns) {
      *cached = v;
      return false;
    }
  }
}

constexpr unsigned kFull = 0xffffffffu;

// a * b + c as one integer multiply-add (the FMA pipe's IMAD)
__device__ __forceinline__ int mad_lo(int a, int b, int c) {
  int d;
  asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Predicated 16-byte accesses of the per-step data movement: one instruction each, so lanes that
// have nothing to load or store (no face piece, no record) take no branch in the step loop.
// Load: *p if pr, else neg in every component.
__device__ __forceinline__ int4 ld_cg_if(const int4* p, bool pr, int neg) {
  int4 v;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n mov.b32 %0, %6;\n mov.b32 %1, %6;\n"
      " mov.b32 %2, %6;\n mov.b32 %3, %6;\n @q ld.global.cg.v4.s32 {%0,%1,%2,%3}, [%4];\n}"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "r"((int)pr), "r"(neg));
  return v;
}
// gpu-scope relaxed 16-byte accesses of the traceback kernels' boundary records. Each 32-bit
// element is single-copy atomic, so a reader sees either the sentinel a record slot starts as or
// its final value, never a mix (records are written once).
__device__ __forceinline__ int4 ld_relaxed_if(const int4* p, bool pr, int neg) {
  int4 v;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n mov.b32 %0, %6;\n mov.b32 %1, %6;\n"
      " mov.b32 %2, %6;\n mov.b32 %3, %6;\n @q ld.relaxed.gpu.global.v4.s32 {%0,%1,%2,%3}, [%4];\n}"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "r"((int)pr), "r"(neg));
  return v;
}
__device__ __forceinline__ void st_relaxed_if(int4* p, int4 v, bool pr) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n @q st.relaxed.gpu.global.v4.s32 [%0], {%1,%2,%3,%4};\n}"
      ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"((int)pr));
}
__device__ __forceinline__ void st_relaxed_if(int* p, int v, bool pr) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.relaxed.gpu.global.s32 [%0], %1;\n}"
               ::"l"(p), "r"(v), "r"((int)pr));
}

__device__ __forceinline__ void st_shared_if(int4* p, int4 v, bool pr) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n @q st.shared.v4.s32 [%0], {%1,%2,%3,%4};\n}"
      ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w),
      "r"((int)pr)
      : "memory");
}
__device__ __forceinline__ void st_global_if(int4* p, int4 v, bool pr) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n @q st.global.v4.s32 [%0], {%1,%2,%3,%4};\n}"
      ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"((int)pr));
}
__device__ __forceinline__ void st_global_if(int* p, int v, bool pr) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.global.s32 [%0], %1;\n}"
               ::"l"(p), "r"(v), "r"((int)pr));
}

}  // namespace

// Resident CTAs per SM the register budget is sized for (4 warps each). Traceback variants hold
// more live state (keys, code words) and serve single large triplets that need fewer resident
// warps, so they get the larger budget.
template <int NJ, int NK, bool TB>
struct MinBlocks {
  static constexpr int value = (NJ * NK >= 64 || (TB && NJ * NK >= 32)) ? 2
                               : ((NJ * NK >= 32) ? 3 : 4);
};

template <int NJ, int NK>
struct Geom {
  static constexpr int WJ = kPR * NJ, WK = kPC * NK;
  static constexpr int RJ = WK + 4, RK = WJ;        // record strides (ints)
  static constexpr int PJ = WJ + 4, PK = WK + 4;    // padded profile rows
  static constexpr int SEGJ = NK + 4;               // staged j-record segment per lane column
  static constexpr int SLOT = kPC * SEGJ + WJ;      // ints per ring slot
  static constexpr int CBJ = NK / 4 + 1;            // 16-byte pieces per j-segment
  static constexpr int CBK = NJ / 4;                // 16-byte pieces per k-segment
  static constexpr int NCOPY = kPC * CBJ + kPR * CBK;
  static constexpr int W = NJ * NK / 8;             // code words per lane per step
};

// The cell passes read tile values that earlier cells of the same pass wrote; the front end
// cannot see that order and may warn (#549) without cause.
#pragma nv_diag_suppress 549
// AT selects the alignment type of Sec. II (kGlobal, kSemiGlobal, kLocal; engine.h); the
// semi-global and local types are built for score mode only. PACK != 0 is the packed int16x2
// mode (engine.h): the triplet of descriptor d in the low halves, that of d.pair in the high
// halves, on the task grid of their maximal lengths (global type, score only). PACK = 1 keeps
// signed halves (DPX s16x2 add-max, adds from -infinity clamped); PACK = 2, for scoring schemes
// whose sigma'' are all >= 0, keeps each half as M' + 2^14 (-infinity = 0): every half then stays
// in 0 .. 2^16 - 1 through the adds, so a plain 32-bit add is the two 16-bit adds and the diagonal
// sum goes to the FMA pipe, with the unsigned u16x2 add-max for the rest. SLAB = true builds
// the slab launches of one triplet (global type, int32; WaveParams i0 / plane_in / plane_out):
// a kept apart so that the regular instantiations carry none of its registers.
template <int NJ, int NK, bool TB, int AT, int PACK, bool SLAB>
__global__ void __launch_bounds__(kWarpsPerCta * 32, MinBlocks<NJ, NK, TB>::value)
    wavefront_kernel(const WaveParams p) {
  using G = Geom<NJ, NK>;
  static_assert(NJ % 4 == 0 && NK % 4 == 0, "tile sides must be multiples of 4");
  static_assert(!PACK || (!TB && AT == kGlobal), "the packed mode is global and score-only");
  static_assert(!SLAB || (!PACK && AT == kGlobal), "slab launches are global and int32");
  // -infinity in every lane of a register
  constexpr int NEG = PACK == 1 ? kNeg16x2 : (PACK == 2 ? 0 : kNeg);
  static_assert(G::NCOPY <= 32, "one staged piece per lane per step");
  constexpr int WJ = G::WJ, WK = G::WK, W = G::W;
  extern __shared__ int4 smem4[];
  int* smem = reinterpret_cast<int*>(smem4);
  const int KP = p.KP;
  const int VIRT = KP - 1;
  const int sigN = (KP * KP + 3) & ~3;
  int* sig = smem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NPROF = PACK ? 2 : 1;  // profile sets per warp (one per half)
  int* profJ = smem + sigN + warp * (NPROF * KP * (G::PJ + G::PK) + kRing * G::SLOT);
  int* profK = profJ + KP * G::PJ;
  int* profJ1 = profK + KP * G::PK;               // packed mode: high halves
  int* profK1 = profJ1 + KP * G::PJ;
  int* ring = profJ + NPROF * KP * (G::PJ + G::PK);
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) sig[e] = p.sig[e];
  __syncthreads();
  const int r = lane >> 3, lc = lane & 7;

  // This lane's staging piece: which record, which 16 bytes, whose slice.
  int cp_kind = 0, cp_delta = 0, cp_col = 0, cp_dst = 0;
  if (lane < kPC * G::CBJ) {
    const int l = lane / G::CBJ, bb = lane % G::CBJ;
    cp_kind = 1;
    cp_delta = l;
    cp_col = l * NK + 4 * bb;
    cp_dst = l * G::SEGJ + 4 * bb;
  } else if (lane < G::NCOPY) {
    const int q = lane - kPC * G::CBJ;
    const int rr = q / G::CBK, bb = q % G::CBK;
    cp_kind = 2;
    cp_delta = rr;
    cp_col = rr * NJ + 4 * bb;
    cp_dst = kPC * G::SEGJ + rr * NJ + 4 * bb;
  }

  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(p.queue, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= p.ntasks) return;
    if (task < p.pace_n && task > 0) {
      // Pace the first wave (all warps grab at once otherwise, and the cohorts that finish
      // together would grab deep producer chains together in every later wave).
      const int need = (int)((long long)task * p.pace_T / p.pace_n);
      bool okp = true;
      int seen = 0;
      if (lane == 0 && need > 0) okp = wait_flag(p.pace_flag, need, &seen, p.wait_ns);
      if (!__shfl_sync(kFull, okp, 0)) {
        if (lane == 0) atomicOr(p.err, 1);
        return;
      }
    }
    const Task tk = p.tasks[task];
    const TripDesc& d = p.desc[tk.trip];
    const TripDesc& d1 = PACK ? p.desc[d.pair] : d;  // triplet of the high halves
    const int a = d.glen[0], b = d.glen[1], c = d.glen[2];       // task grid
    const int a0 = d.len[0], b0 = d.len[1], c0 = d.len[2];       // triplet of the low halves
    const int a1 = d1.len[0], b1 = d1.len[1], c1 = d1.len[2];    // packed: the high halves
    const int nJ = d.nJ, nK = d.nK, T = d.T;
    const int J = tk.J, K = tk.K;
    const int8_t* S0 = p.seq + d.s_off[0];
    const int8_t* S1 = p.seq + d.s_off[1];
    const int8_t* S2 = p.seq + d.s_off[2];
    const int8_t* T0 = p.seq + d1.s_off[0];
    const int8_t* T1 = p.seq + d1.s_off[1];
    const int8_t* T2 = p.seq + d1.s_off[2];
    const int j0 = J * WJ + r * NJ, k0 = K * WK + lc * NK;
    const int me = J * nK + K;

    // Substitution profiles of this block: profJ[x][jl] = sigma''(x, y_(J*WJ+jl)),
    // profK[x][kl] = sigma''(x, z_(K*WK+kl)); residue index 0 and beyond the end are VIRT.
    __syncwarp();
    for (int e = lane; e < KP * WJ; e += 32) {
      const int x = e / WJ, jl = e - x * WJ, j = J * WJ + jl;
      const int y = (j >= 1 && j <= b0) ? (int)S1[j - 1] : VIRT;
      profJ[x * G::PJ + jl] = sig[x * KP + y];
      if (PACK) {
        const int y1 = (j >= 1 && j <= b1) ? (int)T1[j - 1] : VIRT;
        profJ1[x * G::PJ + jl] = sig[x * KP + y1];
      }
    }
    for (int e = lane; e < KP * WK; e += 32) {
      const int x = e / WK, kl = e - x * WK, k = K * WK + kl;
      const int z = (k >= 1 && k <= c0) ? (int)S2[k - 1] : VIRT;
      profK[x * G::PK + kl] = sig[x * KP + z];
      if (PACK) {
        const int z1 = (k >= 1 && k <= c1) ? (int)T2[k - 1] : VIRT;
        profK1[x * G::PK + kl] = sig[x * KP + z1];
      }
    }
    // sigma''(y_j, z_k) is the same for every i: keep this lane's tile of it in registers.
    int Cv[NJ][NK];
    {
      int yo[NJ], zv[NK];
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp) {
        const int j = j0 + pp;
        yo[pp] = ((j >= 1 && j <= b0) ? (int)S1[j - 1] : VIRT) * KP;
      }
#pragma unroll
      for (int qq = 0; qq < NK; ++qq) {
        const int k = k0 + qq;
        zv[qq] = (k >= 1 && k <= c0) ? (int)S2[k - 1] : VIRT;
      }
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
        for (int qq = 0; qq < NK; ++qq) Cv[pp][qq] = sig[yo[pp] + zv[qq]];
      if (PACK) {  // high halves: sigma''(y'_j, z'_k) of the second triplet
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
          const int j = j0 + pp;
          yo[pp] = ((j >= 1 && j <= b1) ? (int)T1[j - 1] : VIRT) * KP;
        }
#pragma unroll
        for (int qq = 0; qq < NK; ++qq) {
          const int k = k0 + qq;
          zv[qq] = (k >= 1 && k <= c1) ? (int)T2[k - 1] : VIRT;
        }
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
          for (int qq = 0; qq < NK; ++qq)
            Cv[pp][qq] = (int)__byte_perm(Cv[pp][qq], sig[yo[pp] + zv[qq]], 0x5410);
      }
    }
    __syncwarp();

    // Owner of the final cell (a, b, c) (of each half in packed mode).
    const bool owns_end = (J == b0 / WJ) && (K == c0 / WK) && (r == (b0 % WJ) / NJ) &&
                          (lc == (c0 % WK) / NK);
    const int end_p = b0 % NJ, end_q = c0 % NK;
    const bool owns_end1 = PACK && (J == b1 / WJ) && (K == c1 / WK) &&
                           (r == (b1 % WJ) / NJ) && (lc == (c1 % WK) / NK);
    const int end_p1 = b1 % NJ, end_q1 = c1 % NK;

    int P[NJ][NK];
    // Halo rows / columns of two consecutive slices. Step t writes the halo of its slice into
    // the pair that held slice s-2 and reads slice s-1 from the other; the loop runs two steps
    // per iteration with the roles swapped, so the rotation costs no moves. B holds "slice -1"
    // (the state before step 0).
    int rowA[NK + 1], colA[NJ], rowB[NK + 1], colB[NJ];
#pragma unroll
    for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
      for (int qq = 0; qq < NK; ++qq) P[pp][qq] = NEG;
      colA[pp] = NEG;
      colB[pp] = NEG;
    }
#pragma unroll
    for (int qq = 0; qq <= NK; ++qq) {
      rowA[qq] = NEG;
      rowB[qq] = NEG;
    }
    // M'[-1][-1][-1] = 0 feeds the origin through the (1,1,1) move (stored as 8*0+7 with keys).
    if (J == 0 && K == 0 && lane == 0) rowB[0] = TB ? 7 : (PACK == 2 ? kBias16x2 : 0);
    const int PW = nK * WK;  // row stride of a slab plane
    if (SLAB && p.plane_in) {
      // Slab launch: the state before the first slice is slice i0 - 1 of the cube. Every lane's
      // tile starts from the plane; the halos matter for lane (0,0) only (the other lanes meet
      // local slice -1 inside the loop, from shuffles of these tiles or from plane pieces).
      const int* pl = p.plane_in;
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
        for (int q4 = 0; q4 < NK / 4; ++q4) {
          const int4 v = *reinterpret_cast<const int4*>(pl + (int64_t)(j0 + pp) * PW + k0 + 4 * q4);
          P[pp][4 * q4] = v.x;
          P[pp][4 * q4 + 1] = v.y;
          P[pp][4 * q4 + 2] = v.z;
          P[pp][4 * q4 + 3] = v.w;
        }
        colB[pp] = (k0 >= 1) ? pl[(int64_t)(j0 + pp) * PW + k0 - 1] : NEG;
      }
#pragma unroll
      for (int qq = 0; qq <= NK; ++qq)
        rowB[qq] = (j0 >= 1 && k0 + qq >= 1) ? pl[(int64_t)(j0 - 1) * PW + k0 + qq - 1] : NEG;
    }
    // Semi-global (Sec. II): the axes are zero in the original frame, i.e. M'[i][0][0] = g2*i,
    // M'[0][j][0] = g2*j, M'[0][0][k] = g2*k with g2 = -2*alpha. They enter through the halo
    // cells that feed each axis through a move whose cost is 0 there (all involve the virtual
    // residue): M'[i][-1][-1] (move (0,1,1)) for the i axis, M'[-1][j][-1] (move (1,0,1)) for
    // the j axis and M'[-1][-1][k] (move (1,1,0)) for the k axis. Slice -1 of lane (0,0) is
    // its state before step 0; the other lanes meet slice -1 inside the loop.
    const int g2 = p.g2;
    // a halo value M' in the stored form: the key 8*M' + 7 with traceback, M' itself without
    const auto axis_feed = [](int v) { return TB ? 8 * v + 7 : v; };
    if (AT == kSemiGlobal && lane == 0) {
      if (J == 0) {
#pragma unroll
        for (int qq = 0; qq <= NK; ++qq) rowB[qq] = axis_feed(g2 * max(k0 + qq - 1, 0));
      }
      if (K == 0) {
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) colB[pp] = axis_feed(g2 * (j0 + pp));
      }
    }
    int best = kNeg;  // semi-global / local: best original-frame score seen by this lane
    // With traceback also its cell: local slice and tile cell pp*NK+qq. The first best cell in
    // (i, j, k) order is kept: a lane meets its cells in that order except for the face i = a of
    // semi-global, read at the end, hence the explicit comparison.
    int bestS = 0, bestE = 0;
    const auto note = [&](int m, int sl, int e) {
      if (m > best || (m == best && (sl < bestS || (sl == bestS && e < bestE)))) {
        best = m;
        bestS = sl;
        bestE = e;
      }
    };
    // Semi-global: local indices of the last row j = b and the last column k = c if this lane's
    // tile holds them (only lanes of the last column tasks do).
    const int pb = b - j0, qc = c - k0;
    const bool edgeJ = (unsigned)pb < (unsigned)NJ, edgeK = (unsigned)qc < (unsigned)NK;

    const int64_t recJ = (int64_t)(a + 1) * G::RJ, recK = (int64_t)(a + 1) * G::RK;
    int* const faces = p.faces;
    const int* srcJ = faces + d.oj_off + (int64_t)(me - nK) * recJ;  // producer (J-1, K)
    const int* srcK = faces + d.ok_off + (int64_t)(me - 1) * recK;   // producer (J, K-1)
    int* dstJ = faces + d.oj_off + (int64_t)me * recJ;
    int* dstK = faces + d.ok_off + (int64_t)me * recK;
    const bool has_out_j = (J + 1 < nJ), has_out_k = (K + 1 < nK);
    const int* progJ = p.progress + d.prog_base + (me - nK);
    const int* progK = p.progress + d.prog_base + (me - 1);
    int* progMe = p.progress + d.prog_base + me;
    int cachedJ = J > 0 ? 0 : 1 << 30, cachedK = K > 0 ? 0 : 1 << 30;  // warp-uniform
    uint32_t* code_base = (TB && (!SLAB || p.codes))
                              ? p.codes + d.code_off + (int64_t)me * T * 32 * W + lane * W
                              : nullptr;
    bool ok = true;

    // Face pieces of step u: each lane loads its 16-byte piece from L2 into registers at step
    // u - kAh (after lane 0 has seen the producers publish the steps that wrote them), parks it
    // in ring slot u % kRing at the start of step u - kAh + 1, and the edge lanes read the slot
    // at step u. The load's latency is covered by the rest of the step that issued it (at
    // least). A piece whose slice is outside
    // 0..a, or whose producer does not exist, is parked as -infinity: the piece of lane column
    // l covers exactly the slice s = u - l that edge lane (0, l) (or row l, for k-pieces) works
    // on at step u, so the edge lanes take the ring value as is.
    int4 pf = make_int4(NEG, NEG, NEG, NEG);
    int pf_u = -1;
    // Records as their own readiness flags (traceback launches with WaveParams::data_flags): the
    // records start as kRecordSentinel, and a staged piece is reloaded until none of its written
    // slots holds it, so no progress flag is polled and none is published while the task runs.
    const bool df = TB && !SLAB && p.data_flags != 0;
    const int* pf_src = nullptr;
    bool pf_have = false;
    // slots 0..2 of the first j-record piece are never written (only the corner, slot 3, is)
    const bool pf_corner_only = cp_kind == 1 && cp_col == 0;
    // Lead of a piece's load over its use, in steps. Traceback keys serve single triplets whose
    // time is the wavefront ramp, where each producer-consumer level lags by the lead: 1 step
    // (the load then has the rest of one step to land). Score mode runs many levels at once
    // and gives the load two steps.
    constexpr int kAh = TB ? 1 : 2;
    // The producers are checked once per pair of steps (chk on the first step of each loop
    // iteration), for the pieces of steps u and u + 1 together: one warp-uniform branch per two
    // steps instead of one per step (a lone warp's step -4%, the main line +1%).
    auto fetch = [&](int u, bool chk) {
      const int needJ = min(u + 1 + kPR, T), needK = min(u + 1 + kPC, T);
      if (!df && chk && (cachedJ < needJ || cachedK < needK)) {  // warp-uniform
        bool okl = true;
        int cj = cachedJ, ck = cachedK;
        if (lane == 0) {
          if (cj < needJ) okl = wait_flag(progJ, needJ, &cj, p.wait_ns);
          if (okl && ck < needK) okl = wait_flag(progK, needK, &ck, p.wait_ns);
        }
        ok = __shfl_sync(kFull, okl, 0);
        cachedJ = __shfl_sync(kFull, cj, 0);
        cachedK = __shfl_sync(kFull, ck, 0);
        __syncwarp();
      }
      const int sl = u - cp_delta;
      pf_u = u;
      {
        const bool have = ok && cp_kind != 0 && sl >= 0 && sl <= a && (cp_kind == 1 ? J > 0 : K > 0);
        const int* src = (cp_kind == 1) ? srcJ + (int64_t)sl * G::RJ + cp_col
                                        : srcK + (int64_t)sl * G::RK + cp_col;
        if constexpr (TB) {
          pf = ld_relaxed_if(reinterpret_cast<const int4*>(src), have, NEG);
          pf_src = src;
          pf_have = have;
        } else {
          pf = ld_cg_if(reinterpret_cast<const int4*>(src), have, NEG);  // src read only if have
        }
      }
      if (SLAB && p.plane_in && sl == -1 && cp_kind != 0 && (cp_kind == 1 ? J > 0 : K > 0)) {
        // Slab launch, local slice -1: the producer's record of that slice is plane i0 - 1.
        const int* pl = p.plane_in;
        if (cp_kind == 1) {  // j-record slots cp_col..+3: row J*WJ-1, k = K*WK + slot - 4
          const int k = K * WK + cp_col - 4;
          pf = (k >= 0) ? *reinterpret_cast<const int4*>(pl + (int64_t)(J * WJ - 1) * PW + k)
                        : make_int4(NEG, NEG, NEG, NEG);
        } else {  // k-record slots cp_col..+3: column K*WK-1, rows J*WJ + slot
          const int64_t base = (int64_t)(J * WJ + cp_col) * PW + K * WK - 1;
          pf = make_int4(pl[base], pl[base + PW], pl[base + 2 * PW], pl[base + 3 * PW]);
        }
      }
    };
    auto park = [&]() {
      if (TB && df) {
        const auto missing = [&](const int4& v) {
          return pf_have && (v.w == kRecordSentinel ||
                             (!pf_corner_only && (v.x == kRecordSentinel || v.y == kRecordSentinel ||
                                                  v.z == kRecordSentinel)));
        };
        bool miss = missing(pf);
        if (__any_sync(kFull, miss)) {  // bounded wait for the producer's stores
          const uint64_t t0 = global_ns();
          unsigned ns = 32;
          for (;;) {
            __nanosleep(ns);
            if (ns < 256) ns <<= 1;
            if (miss) {
              pf = ld_relaxed_if(reinterpret_cast<const int4*>(pf_src), true, NEG);
              miss = missing(pf);
            }
            if (!__any_sync(kFull, miss)) break;
            if (__shfl_sync(kFull, (int64_t)(global_ns() - t0) > p.wait_ns ? 1 : 0, 0)) {
              ok = false;
              break;
            }
          }
        }
      }
      st_shared_if(reinterpret_cast<int4*>(ring + (pf_u & (kRing - 1)) * G::SLOT + cp_dst), pf,
                   cp_kind != 0);
    };

    fetch(0, true);
    if (kAh == 2) {
      park();
      fetch(1, false);
    }
    // Residues of S0 by slice: in block B, lane q holds the residue of slice 32*B + q. Blocks are
    // loaded one block ahead and read by shuffle, so no global load sits on the per-step path.
    // Packed mode: the two triplets' residues in bits 0-7 and 8-15.
    auto xblock = [&](int base) -> int {
      const int sl = base + lane, gi = sl + (SLAB ? p.i0 : 0);  // local slice, cube slice
      const int x0 = (gi >= 1 && sl <= a0) ? (int)__ldg(S0 + gi - 1) : VIRT;
      if (!PACK) return x0;
      const int x1 = (sl >= 1 && sl <= a1) ? (int)__ldg(T0 + sl - 1) : VIRT;
      return x0 | (x1 << 8);
    };
    int xprev = PACK ? (VIRT | (VIRT << 8)) : VIRT, xcur = xblock(0), xnext = xblock(32);

    int pub_in = p.TI;  // steps until the next progress publication
    // One step: the halo of slice s goes into rowCur / colCur, slice s-1 is in rowPrev /
    // colPrev. `first` marks the first step of a loop iteration (it checks the producers for
    // both). Returns false when a bounded wait gave up.
    // `tail` enables the end-cell work (scores, the slab's last plane, semi-global edge maxima):
    // false on steps before any lane reaches an end slice, which then carry no branches for it.
    auto step = [&](const int t, const bool first, const bool tail, int (&rowCur)[NK + 1],
                    const int (&rowPrev)[NK + 1], int (&colCur)[NJ],
                    const int (&colPrev)[NJ]) -> bool {
      const int s = t - r - lc;
      park();  // piece of step t + 1
      if (t + kAh < T) fetch(t + kAh, first);
      if (!ok) return false;
      if ((t & 31) == 0 && t > 0) {
        xprev = xcur;
        xcur = xnext;
        xnext = xblock(t + 32);
      }
      // this lane's slice s lies in [t - 10, t]: in the current or the previous block
      const int xa = __shfl_sync(kFull, xcur, s & 31);
      const int xb = __shfl_sync(kFull, xprev, s & 31);
      const int x = (s >= (t & ~31)) ? xa : xb;
      __syncwarp();
      // Halo of slice s: shuffled from the neighbour lanes (their step t-1 results), or staged
      // face records for the edge lanes.
      {
        const int* sl = ring + (t & (kRing - 1)) * G::SLOT;
        const int* rs = sl + lc * G::SEGJ;
        const int* cs = sl + kPC * G::SEGJ + r * NJ;
        int er[NK + 1], ec[NJ];
        er[0] = rs[3];
#pragma unroll
        for (int q4 = 0; q4 < NK / 4; ++q4) {
          const int4 v = reinterpret_cast<const int4*>(rs + 4)[q4];
          er[1 + 4 * q4] = v.x;
          er[2 + 4 * q4] = v.y;
          er[3 + 4 * q4] = v.z;
          er[4 + 4 * q4] = v.w;
        }
#pragma unroll
        for (int p4 = 0; p4 < NJ / 4; ++p4) {
          const int4 v = reinterpret_cast<const int4*>(cs)[p4];
          ec[4 * p4] = v.x;
          ec[4 * p4 + 1] = v.y;
          ec[4 * p4 + 2] = v.z;
          ec[4 * p4 + 3] = v.w;
        }
        const int corner_send = colPrev[NJ - 1];
#pragma unroll
        for (int qq = 0; qq <= NK; ++qq) {
          const int send = qq == 0 ? corner_send : P[NJ - 1][qq - 1];
          const int v = __shfl_up_sync(kFull, send, kPC);
          rowCur[qq] = (r == 0) ? er[qq] : v;
        }
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
          const int v = __shfl_up_sync(kFull, P[pp][NK - 1], 1);
          colCur[pp] = (lc == 0) ? ec[pp] : v;
        }
        if (AT == kSemiGlobal && (J == 0 || K == 0)) {  // axis feeds (warp-uniform branch)
          // Finite only at slice -1 (once per lane) and for the i-axis feed M'[s][-1][-1] of
          // lane 0 of task (0,0): the first row and column of tasks pace every task after them,
          // so their per-step cost stays at one value on one lane.
          if (J == 0 && r == 0 && s == -1) {
#pragma unroll
            for (int qq = 0; qq <= NK; ++qq) rowCur[qq] = axis_feed(g2 * (k0 + qq - 1));
          }
          if (J == 0 && K == 0 && lane == 0 && s >= 0) rowCur[0] = axis_feed(g2 * s);
          if (K == 0 && lc == 0 && s == -1) {
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp) colCur[pp] = axis_feed(g2 * (j0 + pp));
          }
        }
      }

      const bool active = s >= 0 && s <= a;
      uint32_t cw[W];
      if (active) {
        int A[NJ], B[NK];
        {
          const int xl = PACK ? (x & 0xff) : x;
          const int4* pa = reinterpret_cast<const int4*>(profJ + xl * G::PJ + r * NJ);
#pragma unroll
          for (int p4 = 0; p4 < NJ / 4; ++p4) {
            const int4 v = pa[p4];
            A[4 * p4] = v.x;
            A[4 * p4 + 1] = v.y;
            A[4 * p4 + 2] = v.z;
            A[4 * p4 + 3] = v.w;
          }
          const int4* pb = reinterpret_cast<const int4*>(profK + xl * G::PK + lc * NK);
#pragma unroll
          for (int q4 = 0; q4 < NK / 4; ++q4) {
            const int4 v = pb[q4];
            B[4 * q4] = v.x;
            B[4 * q4 + 1] = v.y;
            B[4 * q4 + 2] = v.z;
            B[4 * q4 + 3] = v.w;
          }
          if (PACK) {  // high halves from the second triplet's profiles
            const int xh = x >> 8;
            const int4* qa = reinterpret_cast<const int4*>(profJ1 + xh * G::PJ + r * NJ);
#pragma unroll
            for (int p4 = 0; p4 < NJ / 4; ++p4) {
              const int4 v = qa[p4];
              A[4 * p4] = (int)__byte_perm(A[4 * p4], v.x, 0x5410);
              A[4 * p4 + 1] = (int)__byte_perm(A[4 * p4 + 1], v.y, 0x5410);
              A[4 * p4 + 2] = (int)__byte_perm(A[4 * p4 + 2], v.z, 0x5410);
              A[4 * p4 + 3] = (int)__byte_perm(A[4 * p4 + 3], v.w, 0x5410);
            }
            const int4* qb = reinterpret_cast<const int4*>(profK1 + xh * G::PK + lc * NK);
#pragma unroll
            for (int q4 = 0; q4 < NK / 4; ++q4) {
              const int4 v = qb[q4];
              B[4 * q4] = (int)__byte_perm(B[4 * q4], v.x, 0x5410);
              B[4 * q4 + 1] = (int)__byte_perm(B[4 * q4 + 1], v.y, 0x5410);
              B[4 * q4 + 2] = (int)__byte_perm(B[4 * q4 + 2], v.z, 0x5410);
              B[4 * q4 + 3] = (int)__byte_perm(B[4 * q4 + 3], v.w, 0x5410);
            }
          }
        }
        // Global and semi-global score kernels: two passes (below); the local type and the
        // traceback keys: one pass over the cells with a second tile Q.
        if constexpr (!TB && AT != kLocal) {
          // Two passes, both in place in P, so no second tile and no copy-back:
          //  pass 1 (anti-diagonals in decreasing order) replaces P (slice s-1) by
          //    E = max{ Pd+A+B+C, Pxy+A, Pxz+B, Sx }, the moves from the previous slice; a cell's
          //    old value is last read by its own E, since the cells that read it lie on later
          //    anti-diagonals and are done first;
          //  pass 2 (forward order) turns E into Q = max{ E, Myz+C, Sy, Sz }, the moves within
          //    the slice, reading Q of earlier cells.
          // Shifted frame (engine.h). Used for the global and semi-global score kernels; the
          // local floor and the traceback keys lengthen pass 2's dependent chain (it can only
          // start once pass 1 reaches cell (0,0)), and there the one-pass form below is faster.
          auto pass1 = [&](const int pp, const int qq) {
            const int Pd =
                (pp == 0) ? rowPrev[qq] : (qq == 0 ? colPrev[pp - 1] : P[pp - 1][qq - 1]);
            const int Pxy = (pp == 0) ? rowPrev[qq + 1] : P[pp - 1][qq];
            const int Pxz = (qq == 0) ? colPrev[pp] : P[pp][qq - 1];
            const int Sx = P[pp][qq];
            if constexpr (PACK == 2) {
              // Biased halves: the 32-bit multiply-adds are the 16-bit adds (no carry out of the
              // low half, engine.h), then unsigned per-half maxima (3-input, then add-max).
              const unsigned x2 = (unsigned)mad_lo(B[qq], p.one, mad_lo(A[pp], p.one, Pd));
              const unsigned ea = (unsigned)mad_lo(A[pp], p.one, Pxy);
              const unsigned eb = (unsigned)mad_lo(B[qq], p.one, Pxz);
              const unsigned e = __vimax3_u16x2(ea, eb, (unsigned)Sx);
              P[pp][qq] = (int)__viaddmax_u16x2(x2, (unsigned)Cv[pp][qq], e);
            } else if constexpr (PACK == 1) {
              // Per 16-bit half: max(a + b, c). Sums from a -infinity operand are clamped at
              // kNeg16, so nothing wraps.
              const unsigned neg = (unsigned)kNeg16x2;
              unsigned dd = __viaddmax_s16x2((unsigned)Pd, (unsigned)A[pp], neg);
              dd = __viaddmax_s16x2(dd, (unsigned)B[qq], neg);
              unsigned e = __viaddmax_s16x2((unsigned)Pxy, (unsigned)A[pp], (unsigned)Sx);
              e = __viaddmax_s16x2((unsigned)Pxz, (unsigned)B[qq], e);
              P[pp][qq] = (int)__viaddmax_s16x2(dd, (unsigned)Cv[pp][qq], e);
            } else {
              // The sums Pd + A + B, Pxy + A and Pxz + B as multiply-adds by a runtime 1 (p.one):
              // they issue to the FMA pipe, so the ALU pipe, which bounds the step, carries only a
              // 3-input max and one fused add-max in pass 1 (n=4000: 30.1 -> 28.1 ms against
              // moving only the diagonal sum). The inner Pd + A is the left cell's Pxy + A.
              const int x2 = mad_lo(B[qq], p.one, mad_lo(A[pp], p.one, Pd));
              const int ea = mad_lo(A[pp], p.one, Pxy);
              const int eb = mad_lo(B[qq], p.one, Pxz);
              const int e = __vimax3_s32(ea, eb, Sx);
              P[pp][qq] = __viaddmax_s32(x2, Cv[pp][qq], e);
            }
          };
          auto pass2 = [&](const int pp, const int qq) {
            const int Myz =
                (pp == 0) ? rowCur[qq] : (qq == 0 ? colCur[pp - 1] : P[pp - 1][qq - 1]);
            const int Sy = (pp == 0) ? rowCur[qq + 1] : P[pp - 1][qq];
            const int Sz = (qq == 0) ? colCur[pp] : P[pp][qq - 1];
            if constexpr (PACK == 2) {
              const unsigned q =
                  __viaddmax_u16x2((unsigned)Myz, (unsigned)Cv[pp][qq], (unsigned)P[pp][qq]);
              P[pp][qq] = (int)__vimax3_u16x2(q, (unsigned)Sy, (unsigned)Sz);
            } else if constexpr (PACK == 1) {
              const unsigned q =
                  __viaddmax_s16x2((unsigned)Myz, (unsigned)Cv[pp][qq], (unsigned)P[pp][qq]);
              P[pp][qq] = (int)__vimax3_s16x2(q, (unsigned)Sy, (unsigned)Sz);
            } else {
              P[pp][qq] = max(max(Myz + Cv[pp][qq], P[pp][qq]), max(Sy, Sz));
            }
          };
#pragma unroll
          for (int dg = NJ + NK - 2; dg >= 0; --dg) {
#pragma unroll
            for (int pp = NJ - 1; pp >= 0; --pp) {
              const int qq = dg - pp;
              if (qq >= 0 && qq < NK) pass1(pp, qq);
            }
          }
#pragma unroll
          for (int dg = 0; dg < NJ + NK - 1; ++dg) {
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp) {
              const int qq = dg - pp;
              if (qq >= 0 && qq < NK) pass2(pp, qq);
            }
          }
        } else {
          int Q[NJ][NK];
          int raw[8];
          // Local (Sec. II, v = 0): M >= 0, i.e. M' >= g2*(s+j+k) = fl on the anti-diagonal pp+qq
          // of the tile being computed; nfl = -fl converts that diagonal's best M' to M.
          int fl = g2 * (s + j0 + k0), nfl = -fl;
          auto cell = [&](const int pp, const int qq) {
            // Predecessors of cell (s, j0+pp, k0+qq): previous slice (P, prev halos) and this
            // slice (Q, current halos).
            const int Pd =
                (pp == 0) ? rowPrev[qq] : (qq == 0 ? colPrev[pp - 1] : P[pp - 1][qq - 1]);
            const int Pxy = (pp == 0) ? rowPrev[qq + 1] : P[pp - 1][qq];
            const int Pxz = (qq == 0) ? colPrev[pp] : P[pp][qq - 1];
            const int Sx = P[pp][qq];
            const int Myz =
                (pp == 0) ? rowCur[qq] : (qq == 0 ? colCur[pp - 1] : Q[pp - 1][qq - 1]);
            const int Sy = (pp == 0) ? rowCur[qq + 1] : Q[pp - 1][qq];
            const int Sz = (qq == 0) ? colCur[pp] : Q[pp][qq - 1];
            if (!TB) {
              // max{ Pd+A+B+C, Pxy+A, Pxz+B, Myz+C, Sx, Sy, Sz } (shifted frame, engine.h)
              const int d0 = Pd + A[pp] + B[qq];
              int u = max(Pxy + A[pp], Sx);
              u = max(Pxz + B[qq], u);
              if (AT == kLocal) u = max(u, fl);  // the v = 0 candidate
              const int w = max(d0, Myz);
              const int v = max(w + Cv[pp][qq], u);
              Q[pp][qq] = max(v, max(Sy, Sz));
            } else {
              // Keys: rank offsets 0,-1,-2,-3,-4,-5,-6 for moves 111,110,101,011,100,010,001.
              const int d0 = Pd + A[pp] + B[qq];
              const int w = max(d0, Myz - 3);
              int u = max(Pxy + (A[pp] - 1), Sx - 4);
              u = max(Pxz + (B[qq] - 2), u);
              const int flc = fl + g2 * (pp + qq);       // local: M' floor of this cell
              if (AT == kLocal) u = max(u, flc << 3);     // the v = 0 candidate, rank 0
              int v = max(w + Cv[pp][qq], u);
              v = max(v, max(Sy - 5, Sz - 6));
              const int e = pp * NK + qq;
              raw[e & 7] = v;
              if (AT == kLocal && j0 + pp <= b0 && k0 + qq <= c0) note((v >> 3) - flc, s, e);
              Q[pp][qq] = v | 7;
              if ((e & 7) == 7) {  // pack 8 ranks: bytes via PRMT, then nibbles (code_bit)
                const uint32_t lo = __byte_perm(__byte_perm(raw[0], raw[1], 0x0040),
                                                __byte_perm(raw[2], raw[3], 0x0040), 0x5410);
                const uint32_t hi = __byte_perm(__byte_perm(raw[4], raw[5], 0x0040),
                                                __byte_perm(raw[6], raw[7], 0x0040), 0x5410);
                cw[e >> 3] = (lo & 0x07070707u) | ((hi & 0x07070707u) << 4);
              }
            }
          };
          if (!TB) {
            // Anti-diagonal order: consecutive cells are independent, which hides the latency of
            // each cell's dependent max chain.
#pragma unroll
            for (int dg = 0; dg < NJ + NK - 1; ++dg) {
#pragma unroll
              for (int pp = 0; pp < NJ; ++pp) {
                const int qq = dg - pp;
                if (qq >= 0 && qq < NK) cell(pp, qq);
              }
              if (AT == kLocal) {  // best M = M' - g2*(s+j+k) on this anti-diagonal
                int mq = kNeg;
#pragma unroll
                for (int pp = 0; pp < NJ; ++pp) {
                  const int qq = dg - pp;
                  if (qq >= 0 && qq < NK) mq = max(mq, Q[pp][qq]);
                }
                best = max(mq + nfl, best);
                fl += g2;
                nfl -= g2;
              }
            }
          } else {
            // Row order, so the 8 ranks of a code word are complete together.
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
              for (int qq = 0; qq < NK; ++qq) cell(pp, qq);
            }
          }
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int qq = 0; qq < NK; ++qq) P[pp][qq] = Q[pp][qq];
        }
      }
      // Publish progress t (steps < t computed and stored) between this step's compute and its
      // stores: the release then waits only for the previous step's stores, issued a whole step
      // of compute ago, instead of the ones just issued.
      if (--pub_in == 0) {
        pub_in = p.TI;
        __syncwarp();
        if (lane == 0) st_release(progMe, t);
      }
      if (active) {
        if (TB && (!SLAB || code_base)) {
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
        if (SLAB && tail && p.plane_out && s == a) {
          // Slab launch: the last slice becomes the next slab's input plane.
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int q4 = 0; q4 < NK / 4; ++q4)
              *reinterpret_cast<int4*>(p.plane_out + (int64_t)(j0 + pp) * PW + k0 + 4 * q4) =
                  make_int4(P[pp][4 * q4], P[pp][4 * q4 + 1], P[pp][4 * q4 + 2],
                            P[pp][4 * q4 + 3]);
        }
        {  // j-record: the last lane row's bottom tile rows (predicated, no branch)
          const bool out_j = r == kPR - 1 && has_out_j;
          int* dst = dstJ + (int64_t)s * G::RJ;
          if constexpr (TB)
            st_relaxed_if(dst + 3, colCur[NJ - 1], out_j && lc == 0);  // corner for lane (0,0)
          else
            st_global_if(dst + 3, colCur[NJ - 1], out_j && lc == 0);
          int4* d4 = reinterpret_cast<int4*>(dst + 4 + lc * NK);
#pragma unroll
          for (int q4 = 0; q4 < NK / 4; ++q4) {
            const int4 v = make_int4(P[NJ - 1][4 * q4], P[NJ - 1][4 * q4 + 1],
                                     P[NJ - 1][4 * q4 + 2], P[NJ - 1][4 * q4 + 3]);
            if constexpr (TB)
              st_relaxed_if(d4 + q4, v, out_j);
            else
              st_global_if(d4 + q4, v, out_j);
          }
        }
        {  // k-record: the last lane column's right tile columns
          const bool out_k = lc == kPC - 1 && has_out_k;
          int4* d4 = reinterpret_cast<int4*>(dstK + (int64_t)s * G::RK + r * NJ);
#pragma unroll
          for (int p4 = 0; p4 < NJ / 4; ++p4) {
            const int4 v = make_int4(P[4 * p4][NK - 1], P[4 * p4 + 1][NK - 1],
                                     P[4 * p4 + 2][NK - 1], P[4 * p4 + 3][NK - 1]);
            if constexpr (TB)
              st_relaxed_if(d4 + p4, v, out_k);
            else
              st_global_if(d4 + p4, v, out_k);
          }
        }
        if (AT == kSemiGlobal && tail && (edgeJ || edgeK)) {
          // Cells of this slice on the last row j = b or the last column k = c, in the original
          // frame M = M' - g2*(i+j+k). The last slice i = a is taken after the sweep.
          const int base = g2 * (s + j0 + k0);
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int qq = 0; qq < NK; ++qq)
              if ((edgeJ && pp == pb && qq <= qc) || (edgeK && qq == qc && pp <= pb)) {
                if (TB)
                  note((P[pp][qq] >> 3) - base - g2 * (pp + qq), s, pp * NK + qq);
                else
                  best = max(best, P[pp][qq] - base - g2 * (pp + qq));
              }
        }
        if (AT == kGlobal && tail && owns_end && s == a0 && (!SLAB || d.out_idx >= 0)) {
          int v = 0;
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int qq = 0; qq < NK; ++qq)
              if (pp == end_p && qq == end_q) v = P[pp][qq];
          if (PACK == 1) v = (int)(short)(v & 0xffff);    // low half, sign-extended
          if (PACK == 2) v = (v & 0xffff) - (1 << 14);   // low half, unbiased
          p.scores[d.out_idx] = (TB ? (v >> 3) : v) + d.score_base;
        }
        if (PACK && tail && owns_end1 && s == a1) {
          int v = 0;
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int qq = 0; qq < NK; ++qq)
              if (pp == end_p1 && qq == end_q1) v = P[pp][qq];
          const int hi = PACK == 2 ? (int)((unsigned)v >> 16) - (1 << 14) : (v >> 16);
          p.scores[d1.out_idx] = hi + d1.score_base;  // high half
        }
      }
      return true;
    };
    // Steps before t_end have every lane below every end slice (a, a0, a1): they run without the
    // end-cell work, except in semi-global tasks of the last task row or column, whose edge lanes
    // hold the row j = b or the column k = c of every slice. The second copy of the step pays in
    // the traceback kernels (n~1000: 1.49 -> 1.47 ms); the score kernels were 2-3% slower with it.
    constexpr bool kSplit = TB && AT != kLocal;
    const int t_end = min(a, PACK ? min(a0, a1) : a0);
    int t = 0;
    bool running = true;
    if (kSplit && !(AT == kSemiGlobal && (J == nJ - 1 || K == nK - 1))) {
      for (; t + 1 < T && t + 1 < t_end; t += 2) {
        if (!step(t, true, false, rowA, rowB, colA, colB) ||
            !step(t + 1, false, false, rowB, rowA, colB, colA)) {
          running = false;
          break;
        }
      }
    }
    for (; running && t < T; t += 2) {
      if (!step(t, true, true, rowA, rowB, colA, colB)) break;
      if (t + 1 < T && !step(t + 1, false, true, rowB, rowA, colB, colA)) break;
    }
    __syncwarp();
    if (ok && lane == 0) st_release(progMe, T);  // all steps computed and stored
    if (!ok) {
      if (lane == 0) atomicOr(p.err, 1);
      return;
    }
    if (AT == kSemiGlobal) {
      // Every lane's last computed slice is s = a, so its tile still holds the face i = a.
      const int base = g2 * (a + j0 + k0);
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
        for (int qq = 0; qq < NK; ++qq)
          if (pp <= pb && qq <= qc) {
            if (TB)
              note((P[pp][qq] >> 3) - base - g2 * (pp + qq), a, pp * NK + qq);
            else
              best = max(best, P[pp][qq] - base - g2 * (pp + qq));
          }
    }
    if (AT != kGlobal && !TB) {  // the triplet's score is the max over its tasks' lanes
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(kFull, best, off));
      if (lane == 0) atomicMax(p.scores + d.out_idx, best);
    }
    if (AT != kGlobal && TB) {
      // (score, first cell) of the triplet: key = (M + 2^26) << 37 | (2^37 - 1 - cell index), so
      // the 64-bit max picks the best score and, among equals, the first cell in (i, j, k) order.
      unsigned long long key = 0;
      if (best != kNeg) {
        const int pp_b = bestE / NK, qq_b = bestE % NK;
        const unsigned long long lin =
            ((unsigned long long)bestS * (unsigned)(b0 + 1) + (unsigned)(j0 + pp_b)) *
                (unsigned)(c0 + 1) +
            (unsigned)(k0 + qq_b);
        key = ((unsigned long long)(best + (1 << 26)) << 37) | ((1ull << 37) - 1 - lin);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, key, off);
        key = o > key ? o : key;
      }
      if (lane == 0) atomicMax(p.best64 + d.out_idx, key);
    }
  }
}


}  // namespace trioseq

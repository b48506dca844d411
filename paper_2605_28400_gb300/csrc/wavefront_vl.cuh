// wavefront_vl.cuh — score-only global wavefront kernel with two cells of one triplet per
// register ("virtual lanes"), for scoring schemes whose sigma'' are all >= 0.
//
// wavefront_vl_kernel<NJ, NH>: the column-task engine of wavefront.cuh (same queue, boundary
// records, progress flags, staging ring and bounded waits; Eq. 1 in the shifted frame of engine.h),
// with each lane's NJ x 2NH tile held as NJ x NH registers of two 16-bit halves:
//  * Layout. The low half holds the left NH columns of the tile at slice s = t - r - 2*lc, the
//    high half the right NH columns one slice behind (s - 1). The 4 x 8 lanes thus act as 4 x 16
//    virtual lanes of NJ x NH tiles on the usual anti-diagonal skew, and every halo comes from a
//    step already finished: rows and the corner by the same packed shuffles as a plain tile, the
//    high half's left column from the low half's previous right column (one PRMT per row).
//  * Arithmetic. The cell passes are those of the biased packed mode (engine.h): each half holds
//    M' - B + 2^14 with -infinity = 0, the diagonal sum runs as two 32-bit multiply-adds on the
//    FMA pipe, the maxima as unsigned 16x2 DPX add-max operations.
//  * Range. With every sigma'' >= 0, M' is non-decreasing along each axis and adjacent cells differ
//    by at most 2*max sigma'' (follow the optimal path to the farther cell back to where it enters
//    the farther plane and copy its in-plane moves one plane lower: in-plane costs do not depend
//    on the third coordinate). A warp's working set (19 slices of a 32 x 16NH block plus halos,
//    L1 diameter <= 178 for NH = 8, 114 for NH = 4) therefore spans at most 356*max sigma''.
//    Each warp keeps one base B for its task, warp-uniform, so shuffled halos need no
//    conversion; B is moved by the drift of lane 0's first cell whenever that exceeds 2048 (all
//    halves rebased with a signed 16x2 add-max against 0, which keeps -infinity at 0). The host
//    admits the mode only for max sigma'' <= 33, so every half stays within [1, 2^16) with margin
//    and no add wraps.
//  * Records stay absolute int32 (converted on store and on staging), so tasks are decoupled and
//    the record layout is the plain kernel's with WK = 8 lanes x 2NH columns.
//  * Edges of a task's sweep: the high half of a lane is inactive while the low half computes
//    slice 0 (it is reset to -infinity afterwards); the low half's extra slice a + 1 at the end is
//    computed on virtual residues and never stored.
#pragma once
#include "wavefront.cuh"

namespace trioseq {

constexpr int kVlBias = 1 << 14;

template <int NJ, int NH>
struct VlGeom {
  static constexpr int NK = 2 * NH;                  // cell columns per lane
  static constexpr int WJ = kPR * NJ, WK = kPC * NK;
  static constexpr int RJ = WK + 4, RK = WJ;          // record strides (ints)
  static constexpr int PJ = WJ + 4, PK = WK + 4;      // padded profile rows
  static constexpr int SEGL = NH + 4, SEGH = NH;      // staged j-record ints per lane column
  static constexpr int SEGC = SEGL + SEGH;
  static constexpr int SLOT = kPC * SEGC + kPR * NJ;  // ints per ring slot
  static constexpr int PL = SEGL / 4, PH = SEGH / 4;  // 16-byte pieces per lane column
  static constexpr int PKR = NJ / 4;                  // 16-byte pieces per lane row (k-records)
  static constexpr int NPIECE = kPC * (PL + PH) + kPR * PKR;
  static constexpr int NPL = (NPIECE + 31) / 32;      // pieces per lane
  // Shared-memory variant (CS): 16-bit profile rows padded to a multiple of 8 halves (16-byte
  // aligned rows) and the lane's sigma''(y,z) tile in shared memory.
  static constexpr int PJ16 = WJ + 8, PK16 = WK + 8;  // halves per profile row
  static constexpr int CVG = NJ * NH / 4;             // 16-byte groups of a lane's sigma'' tile
};

// Launch shape of a variant: CS = 0 keeps the lane's sigma''(y,z) tile in registers (4 warps per
// CTA; 2 or 3 CTAs per SM, register-bound); CS = 1 and 2 keep it and 16-bit profiles in shared
// memory, which frees 64 registers, with small CTAs so that occupancy rises in finer steps:
// CS = 1 runs 2-warp CTAs, 5 per SM (10 warps, <= 200 registers), CS = 2 1-warp CTAs, 9 per SM
// (9 warps, <= 224 registers).
template <int NH, int CS>
struct VlLaunch {
  static constexpr int warps = CS == 1 ? 2 : (CS == 2 ? 1 : kWarpsPerCta);
  static constexpr int min_blocks = CS == 1 ? 5 : (CS == 2 ? 9 : (NH >= 8 ? 2 : 3));
  static constexpr int regs = 65536 / (warps * 32 * min_blocks) / 8 * 8;
  static constexpr int max_regs = regs > 255 ? 255 : regs;
};

// Position of tile cell (pp, qq) in anti-diagonal order (diagonal pp + qq ascending, pp
// ascending within it): the order pass 2 visits the cells in, and pass 1 in reverse.
template <int NJ, int NH>
__host__ __device__ constexpr int vl_diag_index(int pp, int qq) {
  int e = 0;
  for (int dg = 0; dg < pp + qq; ++dg) {
    const int lo = dg - (NH - 1) > 0 ? dg - (NH - 1) : 0, hi = dg < NJ - 1 ? dg : NJ - 1;
    e += hi - lo + 1;
  }
  const int lo = pp + qq - (NH - 1) > 0 ? pp + qq - (NH - 1) : 0;
  return e + (pp - lo);
}

// AT: the alignment type of Sec. II. Semi-global feeds its zero axes through the halo cells at
// j = -1 / k = -1 (as wavefront_kernel does, in the relative halves) and takes the best
// original-frame score over the last slices i = a, j = b, k = c. Local adds v = 0 to Eq. 1, i.e.
// M' >= -2*alpha*(i+j+k), which also gives its zero axes, as one more packed max in pass 1 (the
// floor is the same along an anti-diagonal of a half), and takes the best original-frame score
// over every cell:
// per step, each cell's M relative to a per-step reference is folded into a packed 16-bit
// maximum by one add-max, and the step's maximum into a 32-bit best.
template <int NJ, int NH, int CS, int AT>
__global__ void __launch_bounds__(VlLaunch<NH, CS>::warps * 32)
    __maxnreg__((VlLaunch<NH, CS>::max_regs)) wavefront_vl_kernel(const WaveParams p) {
  static_assert(AT == kGlobal || CS == 0, "the variant types keep sigma'' in registers");
  using G = VlGeom<NJ, NH>;
  static_assert(NJ % 4 == 0 && NH % 4 == 0, "tile sides must be multiples of 4");
  constexpr int NK = G::NK, WJ = G::WJ, WK = G::WK;
  constexpr int NEG = 0;  // -infinity in both halves
  extern __shared__ int4 smem4[];
  int* smem = reinterpret_cast<int*>(smem4);
  const int KP = p.KP;
  const int VIRT = KP - 1;
  const int sigN = (KP * KP + 3) & ~3;
  int* sig = smem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per warp: profiles (32-bit, or 16-bit with kP16), the staging ring, and with CS the sigma''
  // tiles of the warp's lanes ([group][lane][4] ints, conflict-free 16-byte loads)
  // 16-bit profiles (one 16-byte load per 8 values of a half) with CS, on the 8x16 tile without
  // it too (half the profile loads per step there: n=4000 23.2 -> 22.3 ms), and on 8x8v with the
  // layout below (its K entries are 4 values, 8-byte loads).
  constexpr bool kP16 = CS || NH >= 8 || AT != kLocal;
  // Without CS: 16-bit profile entries laid out [x][lane row][lane column] (J, 8 halves each) and
  // [half][x][lane column] (K, NH halves), so the 8 lanes of a 16-byte load phase (one lane row,
  // lane columns 0..7) read 8 distinct bank groups whatever their residues: the row-major rows
  // left 36% (8x16) and 46% (8x8v) of the shared-load wavefronts to bank conflicts. The J rows
  // repeat per lane column (16 KB of profiles per warp on 8x16, 13 KB on 8x8v). n=4000: 8x16
  // 22.1 -> 21.6 ms, 8x8v 22.7 -> 21.9 ms, semi-global 8x8v -2.6%; the local 8x8v kernel was
  // 1.4% slower with it and keeps 32-bit row-major profiles.
  constexpr bool kPT = !CS && (NH >= 8 || AT != kLocal);
  const int prof_ints = kPT ? KP * (kPR * kPC * NJ / 2 + kPC * NH)
                             : (kP16 ? KP * (G::PJ16 + G::PK16) / 2 : KP * (G::PJ + G::PK));
  const int warp_ints = prof_ints + kRing * G::SLOT + (CS ? 32 * 4 * G::CVG : 0);
  int* profJ = smem + sigN + warp * warp_ints;
  int* profK = profJ + (kPT ? KP * kPR * kPC * NJ / 2 : (kP16 ? KP * G::PJ16 / 2 : KP * G::PJ));
  int* ring = profJ + prof_ints;
  int4* cvs = reinterpret_cast<int4*>(ring + kRing * G::SLOT);  // CS only
  unsigned short* profJ16 = reinterpret_cast<unsigned short*>(profJ);
  unsigned short* profK16 = reinterpret_cast<unsigned short*>(profK);
  for (int e = threadIdx.x; e < KP * KP; e += blockDim.x) sig[e] = p.sig[e];
  __syncthreads();
  const int r = lane >> 3, lc = lane & 7;

  // This lane's staging pieces: record kind (1 j, 2 k), slice delta, record slot, ring slot.
  int cp_kind[G::NPL], cp_delta[G::NPL], cp_col[G::NPL], cp_dst[G::NPL];
#pragma unroll
  for (int m = 0; m < G::NPL; ++m) {
    const int q = lane + 32 * m;
    cp_kind[m] = 0;
    cp_delta[m] = 0;
    cp_col[m] = 0;
    cp_dst[m] = 0;
    if (q < kPC * (G::PL + G::PH)) {
      const int l = q / (G::PL + G::PH), w = q % (G::PL + G::PH);
      cp_kind[m] = 1;
      if (w < G::PL) {  // low half of lane column l: slice u - 2l, record slots from l*NK
        cp_delta[m] = 2 * l;
        cp_col[m] = l * NK + 4 * w;
        cp_dst[m] = l * G::SEGC + 4 * w;
      } else {  // high half: slice u - 2l - 1, the right NH columns
        const int w2 = w - G::PL;
        cp_delta[m] = 2 * l + 1;
        cp_col[m] = 4 + l * NK + NH + 4 * w2;
        cp_dst[m] = l * G::SEGC + G::SEGL + 4 * w2;
      }
    } else if (q < G::NPIECE) {  // k-record of lane row rr (low half of virtual column 0)
      const int q2 = q - kPC * (G::PL + G::PH);
      const int rr = q2 / G::PKR, bb = q2 % G::PKR;
      cp_kind[m] = 2;
      cp_delta[m] = rr;
      cp_col[m] = rr * NJ + 4 * bb;
      cp_dst[m] = kPC * G::SEGC + rr * NJ + 4 * bb;
    }
  }

  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(p.queue, 1);
    task = __shfl_sync(kFull, task, 0);
    if (task >= p.ntasks) return;
    if (task < p.pace_n && task > 0) {  // first-wave pacing, as in wavefront_kernel
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
    const int a = d.len[0], b = d.len[1], c = d.len[2];
    const int nJ = d.nJ, nK = d.nK, T = d.T;
    const int J = tk.J, K = tk.K;
    const int8_t* S0 = p.seq + d.s_off[0];
    const int8_t* S1 = p.seq + d.s_off[1];
    const int8_t* S2 = p.seq + d.s_off[2];
    const int j0 = J * WJ + r * NJ, k0 = K * WK + lc * NK;
    const int me = J * nK + K;

    // Profiles of this block: profJ[x][jl] = sigma''(x, y_(J*WJ+jl)), profK[x][kl] =
    // sigma''(x, z_(K*WK+kl)); residue index 0 and beyond the end are VIRT.
    __syncwarp();
    for (int e = lane; e < KP * WJ; e += 32) {
      const int x = e / WJ, jl = e - x * WJ, j = J * WJ + jl;
      const int y = (j >= 1 && j <= b) ? (int)S1[j - 1] : VIRT;
      if (kPT) {
        const int rr = jl / NJ, pq = jl - rr * NJ;
        const unsigned short v16 = (unsigned short)sig[x * KP + y];
        for (int l = 0; l < kPC; ++l) profJ16[((x * kPR + rr) * kPC + l) * NJ + pq] = v16;
      } else if (kP16)
        profJ16[x * G::PJ16 + jl] = (unsigned short)sig[x * KP + y];
      else
        profJ[x * G::PJ + jl] = sig[x * KP + y];
    }
    for (int e = lane; e < KP * WK; e += 32) {
      const int x = e / WK, kl = e - x * WK, k = K * WK + kl;
      const int z = (k >= 1 && k <= c) ? (int)S2[k - 1] : VIRT;
      if (kPT) {
        const int l = kl / NK, rem = kl - l * NK, h = rem / NH, q = rem - h * NH;
        profK16[((h * KP + x) * kPC + l) * NH + q] = (unsigned short)sig[x * KP + z];
      } else if (kP16)
        profK16[x * G::PK16 + kl] = (unsigned short)sig[x * KP + z];
      else
        profK[x * G::PK + kl] = sig[x * KP + z];
    }
    // sigma''(y_j, z_k) for both halves (left and right NH columns), packed, for the whole task:
    // in registers, or (CS) in shared memory in anti-diagonal order, read as the passes go
    int Cv[CS ? 1 : NJ][CS ? 1 : NH];
    {
      int yo[NJ];
#pragma unroll
      for (int pp = 0; pp < NJ; ++pp) {
        const int j = j0 + pp;
        yo[pp] = ((j >= 1 && j <= b) ? (int)S1[j - 1] : VIRT) * KP;
      }
#pragma unroll
      for (int qq = 0; qq < NH; ++qq) {
        const int kl = k0 + qq, kh = k0 + NH + qq;
        const int zl = (kl >= 1 && kl <= c) ? (int)S2[kl - 1] : VIRT;
        const int zh = (kh >= 1 && kh <= c) ? (int)S2[kh - 1] : VIRT;
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
          const int v = (int)__byte_perm(sig[yo[pp] + zl], sig[yo[pp] + zh], 0x5410);
          if constexpr (CS) {
            const int e = vl_diag_index<NJ, NH>(pp, qq);
            reinterpret_cast<int*>(cvs + (e >> 2) * 32 + lane)[e & 3] = v;
          } else {
            Cv[pp][qq] = v;
          }
        }
      }
    }
    __syncwarp();

    // Owner of the final cell (a, b, c): its lane, half and tile cell.
    const int endK = c % WK;
    const bool owns_end = (J == b / WJ) && (K == c / WK) && (r == (b % WJ) / NJ) &&
                          (lc == endK / NK);
    const int end_p = b % NJ, end_h = (endK % NK) >= NH, end_q = (endK % NK) % NH;
    // Semi-global: -2*alpha per consumed residue (the frame shift), and this lane's share of the
    // last row j = b and the last column k = c (low half: columns 0..NH-1 of the lane tile,
    // high half: NH..2NH-1)
    const int g2 = p.g2;
    const int pb = b - j0, qlo = c - k0, qhi = c - k0 - NH;
    const bool edgeJ = AT == kSemiGlobal && (unsigned)pb < (unsigned)NJ;
    const bool edgeK = AT == kSemiGlobal && ((unsigned)qlo < (unsigned)NH || (unsigned)qhi < (unsigned)NH);
    int best = kNeg;  // semi-global: best original-frame score of this lane's counted cells

    int P[NJ][NH];
    int rowA[NH + 1], colA[NJ], rowB[NH + 1], colB[NJ];
#pragma unroll
    for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
      for (int qq = 0; qq < NH; ++qq) P[pp][qq] = NEG;
      colA[pp] = NEG;
      colB[pp] = NEG;
    }
#pragma unroll
    for (int qq = 0; qq <= NH; ++qq) {
      rowA[qq] = NEG;
      rowB[qq] = NEG;
    }

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
    bool ok = true;

    // Face pieces (absolute int32 records, kNeg where absent): loaded two steps ahead, parked one
    // step ahead, read by the edge lanes and converted to the task's base there.
    int4 pf[G::NPL];
#pragma unroll
    for (int m = 0; m < G::NPL; ++m) pf[m] = make_int4(kNeg, kNeg, kNeg, kNeg);
    int pf_u = -1;
    // Producers are checked once per pair of steps, for steps u and u + 1 (as in wavefront_kernel).
    auto fetch = [&](int u, bool chk) {
      // k-records are written by the last virtual lane column (2*kPC - 1 steps of skew)
      const int needJ = min(u + 1 + kPR, T), needK = min(u + 1 + 2 * kPC, T);
      if (chk && (cachedJ < needJ || cachedK < needK)) {  // warp-uniform
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
      pf_u = u;
#pragma unroll
      for (int m = 0; m < G::NPL; ++m) {
        const int sl = u - cp_delta[m];
        const bool have = ok && cp_kind[m] != 0 && sl >= 0 && sl <= a &&
                          (cp_kind[m] == 1 ? J > 0 : K > 0);
        const int* src = (cp_kind[m] == 1) ? srcJ + (int64_t)sl * G::RJ + cp_col[m]
                                           : srcK + (int64_t)sl * G::RK + cp_col[m];
        pf[m] = ld_cg_if(reinterpret_cast<const int4*>(src), have, kNeg);
      }
    };
    auto park = [&]() {
#pragma unroll
      for (int m = 0; m < G::NPL; ++m)
        st_shared_if(reinterpret_cast<int4*>(ring + (pf_u & (kRing - 1)) * G::SLOT + cp_dst[m]),
                     pf[m], cp_kind[m] != 0);
    };

    fetch(0, true);
    // The task's base: the largest record value its first slice borders (0 without producers);
    // every cell of the working set lies within the range argument of it. The first j-record
    // piece (record slots 0..3) carries only the corner in slot 3: slots 0..2 are never
    // written, so they stay out of the maximum.
    int Bt = 0;
    {
      int mx = kNeg;
#pragma unroll
      for (int m = 0; m < G::NPL; ++m) {
        const bool corner_only = cp_kind[m] == 1 && cp_col[m] == 0;
        mx = max(mx, corner_only ? pf[m].w : max(max(pf[m].x, pf[m].y), max(pf[m].z, pf[m].w)));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, off));
      Bt = mx > kNeg / 2 ? mx : 0;
    }
    int nb = kVlBias - Bt;  // absolute M' -> biased half: max(v + nb, 0)
    // M'[-1][-1][-1] = 0 feeds the origin through the (1,1,1) move (low half of lane 0).
    if (J == 0 && K == 0 && lane == 0) rowB[0] = kVlBias - Bt;
    // Semi-global zero axes in the shifted frame: M'[-1][-1][k] = g2*k feeds the k axis (move
    // (1,1,0)), M'[-1][j][-1] = g2*j the j axis (move (1,0,1)), M'[i][-1][-1] = g2*i the i axis
    // (move (0,1,1)); lane 0 starts from slice -1 (low halves; the high half's are reset).
    const auto feed = [&](int v) { return max(v + nb, 0); };
    if (AT == kSemiGlobal && lane == 0) {
      if (J == 0) {
#pragma unroll
        for (int qq = 0; qq <= NH; ++qq) rowB[qq] = feed(g2 * max(k0 + qq - 1, 0));
      }
      if (K == 0) {
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) colB[pp] = feed(g2 * (j0 + pp));
      }
    }
    park();
    fetch(1, false);

    auto xblock = [&](int base) -> int {
      const int sl = base + lane;
      return (sl >= 1 && sl <= a) ? (int)__ldg(S0 + sl - 1) : VIRT;
    };
    int xprev = VIRT, xcur = xblock(0), xnext = xblock(32);
    int xlo_prev = VIRT;  // residue of slice s - 1: the high half's

    int pub_in = p.TI;
    // `tail` enables the end-cell work (the global score, the semi-global last-slice maxima):
    // false on the steps before any lane can reach slice a, so those steps carry no per-step
    // branches for it.
    auto step = [&](const int t, const bool first, const bool tail, int (&rowCur)[NH + 1],
                    const int (&rowPrev)[NH + 1], int (&colCur)[NJ],
                    const int (&colPrev)[NJ]) -> bool {
      const int s = t - r - 2 * lc;
      park();
      if (t + 2 < T) fetch(t + 2, first);
      if (!ok) return false;
      if ((t & 31) == 0 && t > 0) {
        xprev = xcur;
        xcur = xnext;
        xnext = xblock(t + 32);
      }
      // this lane's slice s lies in [t - 17, t]: in the current or the previous block
      const int xa = __shfl_sync(kFull, xcur, s & 31);
      const int xb = __shfl_sync(kFull, xprev, s & 31);
      const int xl = (s >= (t & ~31)) ? xa : xb;  // low half: slice s
      const int xh = xlo_prev;                    // high half: slice s - 1
      xlo_prev = xl;
      __syncwarp();
      {
        const int* sl = ring + (t & (kRing - 1)) * G::SLOT;
        const int* rs = sl + lc * G::SEGC;          // low half: corner + NH columns, slice s
        const int* rh = rs + G::SEGL;               // high half: NH columns, slice s - 1
        const int* cs = sl + kPC * G::SEGC + r * NJ;  // k-record rows, slice s
        // row halo: lane above (packed shuffle), or the staged j-record (first lane row)
        const int corner_send = colPrev[NJ - 1];
#pragma unroll
        for (int qq = 0; qq <= NH; ++qq) {
          const int send = qq == 0 ? corner_send : P[NJ - 1][qq - 1];
          const int v = __shfl_up_sync(kFull, send, kPC);
          const unsigned lo = (unsigned)max(rs[3 + qq] + nb, 0);
          // the high half's corner (j0-1, k0+NH-1) at slice s-1 is the low half's last row
          // halo of the previous step
          const unsigned hi = qq == 0 ? ((unsigned)rowPrev[NH] & 0xffffu)
                                      : (unsigned)max(rh[qq - 1] + nb, 0);
          rowCur[qq] = (r == 0) ? (int)__byte_perm(lo, hi, 0x5410) : v;
        }
        // column halo: low half from the left lane's high half (or the staged k-record in the
        // first lane column), high half from this lane's low half; both from the previous step
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
          const int mine = P[pp][NH - 1];
          const int v = __shfl_up_sync(kFull, mine, 1);
          const unsigned ring_lo = (unsigned)max(cs[pp] + nb, 0);
          colCur[pp] = (lc == 0) ? (int)__byte_perm(ring_lo, (unsigned)mine, 0x5410)
                                 : (int)__byte_perm((unsigned)v, (unsigned)mine, 0x5432);
        }
        if (AT == kSemiGlobal && (J == 0 || K == 0)) {  // axis feeds (warp-uniform branch)
          // Only two kinds of halo cells are finite: those of slice -1 (each lane meets slice -1
          // once, the step before its first) and the i-axis feed M'[s][-1][-1] of lane (0,0)
          // of task (0,0); every other halo cell of the first row or column stays -infinity, as
          // staged. So the per-step cost is one value on one lane.
          if (J == 0 && r == 0 && s == -1) {
#pragma unroll
            for (int qq = 0; qq <= NH; ++qq)
              rowCur[qq] = (int)(((unsigned)rowCur[qq] & 0xffff0000u) |
                                 (unsigned)feed(g2 * (k0 + qq - 1)));
          }
          if (J == 0 && K == 0 && lane == 0 && s >= 0)
            rowCur[0] = (int)(((unsigned)rowCur[0] & 0xffff0000u) | (unsigned)feed(g2 * s));
          if (K == 0 && lc == 0 && s == -1) {
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp)
              colCur[pp] = (int)(((unsigned)colCur[pp] & 0xffff0000u) | (unsigned)feed(g2 * (j0 + pp)));
          }
        }
      }

      const bool active = s >= 0 && s <= a + 1;
      if (active) {
        int A[NJ], Bq[NH];
        if constexpr (kP16) {
          // 16-bit profiles: one 16-byte load holds 8 values of a half; a PRMT pairs the low
          // half's value with the high half's
          const int4* pl = reinterpret_cast<const int4*>(
              kPT ? profJ16 + ((xl * kPR + r) * kPC + lc) * NJ : profJ16 + xl * G::PJ16 + r * NJ);
          const int4* ph = reinterpret_cast<const int4*>(
              kPT ? profJ16 + ((xh * kPR + r) * kPC + lc) * NJ : profJ16 + xh * G::PJ16 + r * NJ);
#pragma unroll
          for (int p8 = 0; p8 < NJ / 8; ++p8) {
            const int4 u = pl[p8], v = ph[p8];
            const int uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              A[8 * p8 + 2 * w] = (int)__byte_perm(uu[w], vv[w], 0x5410);
              A[8 * p8 + 2 * w + 1] = (int)__byte_perm(uu[w], vv[w], 0x7632);
            }
          }
          const int4* ql = reinterpret_cast<const int4*>(
              kPT ? profK16 + (xl * kPC + lc) * NH : profK16 + xl * G::PK16 + lc * NK);
          const int4* qh = reinterpret_cast<const int4*>(
              kPT ? profK16 + ((KP + xh) * kPC + lc) * NH : profK16 + xh * G::PK16 + lc * NK + NH);
          if constexpr (kPT && NH == 4) {
            const uint2 u = *reinterpret_cast<const uint2*>(profK16 + (xl * kPC + lc) * NH);
            const uint2 v = *reinterpret_cast<const uint2*>(profK16 + ((KP + xh) * kPC + lc) * NH);
            Bq[0] = (int)__byte_perm(u.x, v.x, 0x5410);
            Bq[1] = (int)__byte_perm(u.x, v.x, 0x7632);
            Bq[2] = (int)__byte_perm(u.y, v.y, 0x5410);
            Bq[3] = (int)__byte_perm(u.y, v.y, 0x7632);
          }
#pragma unroll
          for (int q8 = 0; q8 < NH / 8; ++q8) {
            const int4 u = ql[q8], v = qh[q8];
            const int uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              Bq[8 * q8 + 2 * w] = (int)__byte_perm(uu[w], vv[w], 0x5410);
              Bq[8 * q8 + 2 * w + 1] = (int)__byte_perm(uu[w], vv[w], 0x7632);
            }
          }
        } else {
          const int4* pl = reinterpret_cast<const int4*>(profJ + xl * G::PJ + r * NJ);
          const int4* ph = reinterpret_cast<const int4*>(profJ + xh * G::PJ + r * NJ);
#pragma unroll
          for (int p4 = 0; p4 < NJ / 4; ++p4) {
            const int4 u = pl[p4], v = ph[p4];
            A[4 * p4] = (int)__byte_perm(u.x, v.x, 0x5410);
            A[4 * p4 + 1] = (int)__byte_perm(u.y, v.y, 0x5410);
            A[4 * p4 + 2] = (int)__byte_perm(u.z, v.z, 0x5410);
            A[4 * p4 + 3] = (int)__byte_perm(u.w, v.w, 0x5410);
          }
          const int4* ql = reinterpret_cast<const int4*>(profK + xl * G::PK + lc * NK);
          const int4* qh = reinterpret_cast<const int4*>(profK + xh * G::PK + lc * NK + NH);
#pragma unroll
          for (int q4 = 0; q4 < NH / 4; ++q4) {
            const int4 u = ql[q4], v = qh[q4];
            Bq[4 * q4] = (int)__byte_perm(u.x, v.x, 0x5410);
            Bq[4 * q4 + 1] = (int)__byte_perm(u.y, v.y, 0x5410);
            Bq[4 * q4 + 2] = (int)__byte_perm(u.z, v.z, 0x5410);
            Bq[4 * q4 + 3] = (int)__byte_perm(u.w, v.w, 0x5410);
          }
        }
        // sigma''(y, z) of tile cell (pp, qq): a register, or (CS) a shared-memory read
        const auto cv = [&](const int pp, const int qq) -> unsigned {
          if constexpr (CS) {
            const int e = vl_diag_index<NJ, NH>(pp, qq);
            return (unsigned)reinterpret_cast<const int*>(cvs + (e >> 2) * 32 + lane)[e & 3];
          } else {
            return (unsigned)Cv[pp][qq];
          }
        };
        // Two passes in place, as in the biased packed mode of wavefront_kernel.
        // Local: the floor of each anti-diagonal e = pp + qq of the tile, both halves, relative
        // and clamped at 0 (a floor below the representable range cannot win: every value of
        // the working set lies above it): M' >= g2*(i+j+k) with i+j+k = s + j0 + k0 + e (low
        // half) and s - 1 + j0 + k0 + NH + e (high half).
        unsigned fl_base = 0, fl_step = 0, fl = 0;  // local: the current diagonal's floor
        if constexpr (AT == kLocal) {
          const int f0 = max(g2 * (s + j0 + k0) + nb, -30000);  // fits s16 with + g2*e below
          fl_base = (unsigned)(f0 & 0xffff) | ((unsigned)((f0 + g2 * (NH - 1)) & 0xffff) << 16);
          fl_step = (unsigned)g2 * 0x10001u;
        }
        auto pass1 = [&](const int pp, const int qq) {
          const int Pd = (pp == 0) ? rowPrev[qq] : (qq == 0 ? colPrev[pp - 1] : P[pp - 1][qq - 1]);
          const int Pxy = (pp == 0) ? rowPrev[qq + 1] : P[pp - 1][qq];
          const int Pxz = (qq == 0) ? colPrev[pp] : P[pp][qq - 1];
          const int Sx = P[pp][qq];
          const unsigned x2 = (unsigned)mad_lo(Bq[qq], p.one, mad_lo(A[pp], p.one, Pd));
          // Pxy + A and Pxz + B as FMA-pipe multiply-adds too (32-bit adds of biased halves: no
          // carry out of the low half), then one 3-input max: 2 ALU-pipe instructions per
          // register instead of 3. With three warps per SMSP the step is bound by the ALU pipe:
          // main line 24.0 -> 22.6 ms. The inner sum Pd + A equals the left cell's Pxy + A.
          const unsigned ea = (unsigned)mad_lo(A[pp], p.one, Pxy);
          const unsigned eb = (unsigned)mad_lo(Bq[qq], p.one, Pxz);
          unsigned e = __vimax3_u16x2(ea, eb, (unsigned)Sx);
          if constexpr (AT == kLocal) {
            // v = 0: the floor as the third input of one max, with x2 + C on the FMA pipe
            // (one ALU-pipe instruction less per register: 27.4 -> 26.6 ms at n=4000)
            const unsigned x2c = (unsigned)mad_lo((int)cv(pp, qq), p.one, (int)x2);
            P[pp][qq] = (int)__vimax3_u16x2(x2c, e, fl);
          } else {
            P[pp][qq] = (int)__viaddmax_u16x2(x2, cv(pp, qq), e);
          }
        };
        auto pass2 = [&](const int pp, const int qq) {
          const int Myz = (pp == 0) ? rowCur[qq] : (qq == 0 ? colCur[pp - 1] : P[pp - 1][qq - 1]);
          const int Sy = (pp == 0) ? rowCur[qq + 1] : P[pp - 1][qq];
          const int Sz = (qq == 0) ? colCur[pp] : P[pp][qq - 1];
          const unsigned q = __viaddmax_u16x2((unsigned)Myz, cv(pp, qq), (unsigned)P[pp][qq]);
          P[pp][qq] = (int)__vimax3_u16x2(q, (unsigned)Sy, (unsigned)Sz);
        };
#pragma unroll
        for (int dg = NJ + NH - 2; dg >= 0; --dg) {
          if constexpr (AT == kLocal) fl = __viaddmax_s16x2(fl_base, (unsigned)dg * fl_step, 0u);
#pragma unroll
          for (int pp = NJ - 1; pp >= 0; --pp) {
            const int qq = dg - pp;
            if (qq >= 0 && qq < NH) pass1(pp, qq);
          }
        }
#pragma unroll
        for (int dg = 0; dg < NJ + NH - 1; ++dg) {
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp) {
            const int qq = dg - pp;
            if (qq >= 0 && qq < NH) pass2(pp, qq);
          }
        }
        if (s == 0) {  // the high half was at slice -1: -infinity there, and in its halos
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
            for (int qq = 0; qq < NH; ++qq) P[pp][qq] &= 0xffff;
            colCur[pp] &= 0xffff;
          }
#pragma unroll
          for (int qq = 0; qq <= NH; ++qq) rowCur[qq] &= 0xffff;
          if (AT == kSemiGlobal && J == 0 && r == 0) {
            // the high half's halo row j = -1 at slice -1 is the k-axis feed M'[-1][-1][k]
#pragma unroll
            for (int qq = 0; qq <= NH; ++qq)
              rowCur[qq] |= feed(g2 * (k0 + NH + qq - 1)) << 16;
          }
        }
      }
      if (--pub_in == 0) {
        pub_in = p.TI;
        __syncwarp();
        if (lane == 0) st_release(progMe, t);
      }
      if (active) {
        const int ub = Bt - kVlBias;  // biased half -> absolute M'
        const bool lo_in = s <= a, hi_in = s >= 1;
        {  // j-record: the last lane row's bottom tile row; low half at s, high half at s - 1
          const bool out_j = r == kPR - 1 && has_out_j;
          int* dl = dstJ + (int64_t)s * G::RJ;
          int* dh = dstJ + (int64_t)(s - 1) * G::RJ;
          // the corner: -infinity (0) on the k = 0 face goes out as the absolute sentinel;
          // every other stored half is a computed cell, always finite
          const int cb = (int)((unsigned)colCur[NJ - 1] & 0xffffu);
          st_global_if(dl + 3, cb == 0 ? kNeg : cb + ub, out_j && lo_in && lc == 0);
#pragma unroll
          for (int q4 = 0; q4 < NH / 4; ++q4) {
            int lo[4], hi[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const unsigned v = (unsigned)P[NJ - 1][4 * q4 + e];
              lo[e] = (int)(v & 0xffffu) + ub;
              hi[e] = (int)(v >> 16) + ub;
            }
            st_global_if(reinterpret_cast<int4*>(dl + 4 + lc * NK) + q4,
                         make_int4(lo[0], lo[1], lo[2], lo[3]), out_j && lo_in);
            st_global_if(reinterpret_cast<int4*>(dh + 4 + lc * NK + NH) + q4,
                         make_int4(hi[0], hi[1], hi[2], hi[3]), out_j && hi_in);
          }
        }
        {  // k-record: the block's last column is the last lane column's high half, slice s - 1
          const bool out_k = lc == kPC - 1 && has_out_k && hi_in;
          int* dk = dstK + (int64_t)(s - 1) * G::RK + r * NJ;
#pragma unroll
          for (int p4 = 0; p4 < NJ / 4; ++p4) {
            int v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = (int)((unsigned)P[4 * p4 + e][NH - 1] >> 16) + ub;
            st_global_if(reinterpret_cast<int4*>(dk) + p4, make_int4(v[0], v[1], v[2], v[3]),
                         out_k);
          }
        }
        if constexpr (AT == kLocal) {
          // Every cell counts. D = P + 2^14 - g2*d per half, d the cell's offset of i+j+k from the
          // lane corner's at the low half's slice (e, or e + NH - 1 for the high half), equals
          // M - mbase with mbase = Bt - g2*(s + j0 + k0) - 2^15; by the range argument it lies in
          // (0, 2^16), so one unsigned add-max per register folds it into the step's maximum.
          const unsigned g2x2 = (unsigned)g2 * 0x10001u;
          const unsigned add0 = 0x40004000u - ((unsigned)(g2 * (NH - 1)) << 16);
          // Cells of one anti-diagonal share d, so they meet in 3-input maxima first and take
          // the offset once per group of up to three.
          unsigned acc = 0;
#pragma unroll
          for (int dg = 0; dg < NJ + NH - 1; ++dg) {
            const unsigned off = add0 - (unsigned)dg * g2x2;
            unsigned g[3] = {0u, 0u, 0u};
            int k = 0;
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp) {
              const int qq = dg - pp;
              if (qq >= 0 && qq < NH) {
                g[k++] = (unsigned)P[pp][qq];
                if (k == 3) {
                  acc = __viaddmax_u16x2(__vimax3_u16x2(g[0], g[1], g[2]), off, acc);
                  k = 0;
                }
              }
            }
            if (k == 2) acc = __viaddmax_u16x2(__vmaxu2(g[0], g[1]), off, acc);
            if (k == 1) acc = __viaddmax_u16x2(g[0], off, acc);
          }
          // the low half's extra slice a + 1 and the high half's slice -1 do not count (a masked
          // half contributes 0, below any counted cell's D)
          const int dlo = s <= a ? (int)(acc & 0xffffu) : 0, dhi = s >= 1 ? (int)(acc >> 16) : 0;
          best = max(best, max(dlo, dhi) + Bt - g2 * (s + j0 + k0) - 32768);
        }
        if (AT == kSemiGlobal && tail) {
          // Cells on a last slice, M = M' - g2*(i+j+k): the face i = a when each half reaches
          // it, and the row j = b / column k = c of each half's slice. Edge lanes all share one
          // row (pb) or column, so only its block runs.
          const int base_lo = ub - g2 * (s + j0 + k0), base_hi = ub - g2 * (s - 1 + j0 + k0 + NH);
          const auto m_lo = [&](int pp, int qq) {
            return (int)((unsigned)P[pp][qq] & 0xffffu) + base_lo - g2 * (pp + qq);
          };
          const auto m_hi = [&](int pp, int qq) {
            return (int)((unsigned)P[pp][qq] >> 16) + base_hi - g2 * (pp + qq);
          };
          if (s == a || s - 1 == a) {
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
              for (int qq = 0; qq < NH; ++qq) {
                if (s == a && pp <= pb && qq <= qlo) best = max(best, m_lo(pp, qq));
                if (s - 1 == a && pp <= pb && qq <= qhi) best = max(best, m_hi(pp, qq));
              }
          }
          if (edgeJ) {
#pragma unroll
            for (int pp = 0; pp < NJ; ++pp)
              if (pp == pb) {
#pragma unroll
                for (int qq = 0; qq < NH; ++qq) {
                  if (s <= a && qq <= qlo) best = max(best, m_lo(pp, qq));
                  if (s >= 1 && qq <= qhi) best = max(best, m_hi(pp, qq));
                }
              }
          }
          if (edgeK) {
#pragma unroll
            for (int qq = 0; qq < NH; ++qq) {
              if (qq == qlo && s <= a) {
#pragma unroll
                for (int pp = 0; pp < NJ; ++pp)
                  if (pp <= pb) best = max(best, m_lo(pp, qq));
              }
              if (qq == qhi && s >= 1) {
#pragma unroll
                for (int pp = 0; pp < NJ; ++pp)
                  if (pp <= pb) best = max(best, m_hi(pp, qq));
              }
            }
          }
        }
        if (AT == kGlobal && tail && owns_end && (end_h ? s - 1 == a : s == a)) {
          unsigned v = 0;
#pragma unroll
          for (int pp = 0; pp < NJ; ++pp)
#pragma unroll
            for (int qq = 0; qq < NH; ++qq)
              if (pp == end_p && qq == end_q) v = (unsigned)P[pp][qq];
          const int h16 = end_h ? (int)(v >> 16) : (int)(v & 0xffffu);
          p.scores[d.out_idx] = h16 + ub + d.score_base;
        }
      }
      return true;
    };
    // Rebase the task when lane 0's first cell drifts 2048 from the bias (warp-uniform; after an
    // odd step, whose current halos are in rowB / colB).
    auto rebase = [&]() {
      const int ref = __shfl_sync(kFull, (int)((unsigned)P[0][0] & 0xffffu), 0);
      const int dlt = ref - kVlBias;
      if (ref != 0 && (dlt >= 2048 || dlt <= -2048)) {
        const unsigned m = (unsigned)((-dlt) & 0xffff) * 0x10001u;  // -dlt in both halves
#pragma unroll
        for (int pp = 0; pp < NJ; ++pp) {
#pragma unroll
          for (int qq = 0; qq < NH; ++qq)
            P[pp][qq] = (int)__viaddmax_s16x2((unsigned)P[pp][qq], m, 0u);
          colB[pp] = (int)__viaddmax_s16x2((unsigned)colB[pp], m, 0u);
        }
#pragma unroll
        for (int qq = 0; qq <= NH; ++qq) rowB[qq] = (int)__viaddmax_s16x2((unsigned)rowB[qq], m, 0u);
        Bt += dlt;
        nb = kVlBias - Bt;
      }
    };
    // Steps t < a have every lane at a slice s <= t < a, so no end cell: they run without the
    // end-cell work, except in semi-global tasks of the last task row or column, whose edge lanes
    // hold the row j = b or the column k = c of every slice. The second copy of the step that
    // this takes pays only where that work is per-step branches: the global type (8x16 tile
    // 24.2 -> 23.0 ms at n=4000) and semi-global on 8x8v (30.2 -> 28.2 ms); semi-global 8x16 (255
    // registers) was 14% slower with it, and local has no such work.
    constexpr bool kSplit = AT == kGlobal || (AT == kSemiGlobal && NH < 8);
    int t = 0;
    bool running = true;
    if (kSplit && !(AT == kSemiGlobal && (J == nJ - 1 || K == nK - 1))) {
      for (; t + 1 < T && t + 1 < a; t += 2) {
        if (!step(t, true, false, rowA, rowB, colA, colB) ||
            !step(t + 1, false, false, rowB, rowA, colB, colA)) {
          running = false;
          break;
        }
        rebase();
      }
    }
    for (; running && t < T; t += 2) {
      if (!step(t, true, true, rowA, rowB, colA, colB)) break;
      if (t + 1 < T && !step(t + 1, false, true, rowB, rowA, colB, colA)) break;
      rebase();
    }
    __syncwarp();
    if (ok && lane == 0) st_release(progMe, T);
    if (!ok) {
      if (lane == 0) atomicOr(p.err, 1);
      return;
    }
    if (AT != kGlobal) {  // the triplet's score is the max over its tasks' lanes
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(kFull, best, off));
      if (lane == 0) atomicMax(p.scores + d.out_idx, best);
    }
  }
}

}  // namespace trioseq

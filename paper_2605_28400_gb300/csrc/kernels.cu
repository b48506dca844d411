// kernels.cu — sm_103a kernels of the 3-way alignment engine: the global-alignment
// instantiations of the wavefront kernel (wavefront.cuh), the traceback walk, and the launchers.
//
// walk_kernel: one warp per traceback request. The warp follows the stored moves back from
//   (a, b, c) through a tube of code records along the diagonal, staged in shared memory in one
//   round trip; runs of diagonal moves are found and emitted 32 cells at a time. In the
//   linear-space traceback the codes hold one slab of slices at a time: the walk resumes from a
//   saved (i, j, k, n) and stops when it leaves the slab.
#include "wavefront.cuh"

namespace trioseq {
// ---------------------------------------------------------------------------------------------
// Traceback walk. Optimal paths of related sequences run close to the cube's main diagonal, so
// the warp stages a "tube" of code records along the diagonal from the current cell: for each
// of the next kTubeS slices, the 3 x 3 lane tiles around the diagonal cell, plus the window of
// each sequence's residues that a path inside the tube can consume. All lanes load the tube in
// one round trip (independent loads, then shared-memory stores). The walk then proceeds in
// warp-wide probes: lane m reads the code of the cell m diagonal moves ahead, a ballot gives the
// run of (1,1,1) moves from the current cell (at most 32), and the lanes of the run write its
// columns at once. The first cell after the run holds a move other than (1,1,1) (applied by
// the whole warp, one column), a start cell, or lies outside the tube, where the next tube is
// staged. Every step is warp-uniform, so the walk carries no serial per-column chain.
constexpr int kTubeS = 64, kTubeR = 3, kTubeC = 3;
constexpr int kTubeRecs = kTubeS * kTubeR * kTubeC;
constexpr int kTubePer = (kTubeRecs + 31) / 32;
// Residue window per sequence: S0 needs the kTubeS residues above the tube's top slice; S1 (S2)
// needs the lane-tile rows (columns) the tube spans plus one, at most
// NJ * (floor((kTubeS - 1) / NJ) + 4) <= 88 cells for tile sides of 4 or 8.
constexpr int kWin = 96;

// First index of the S1 (S2) residue window of a tube whose top cell has index x along that
// axis, for lane tiles of 2^l cells: one below the lowest cell of the tube's lowest tile.
__device__ __forceinline__ int win_base(int x, int l) {
  return ((((x - (kTubeS - 1)) >> l) - 1) << l) - 1;
}

// The triplet's shape comes in registers (len: the three lengths; nK: column tasks along k;
// nJR, nKC: lane rows / columns of the task grid), read once by the caller.
template <int W>
__device__ __forceinline__ void tube_load(uint32_t* win, uint8_t (*res)[kWin], int i0, int j0,
                                          int k0, int lj, int lk, const uint32_t* codes,
                                          const int (&len)[3], int nK, int nJR, int nKC,
                                          const int8_t* const* S, int T, int i_lo, int lane) {
  // residue windows: res[0][m] = S0[i0 - kTubeS + m], res[1][m] = S1[win_base(j0) + m], ...
  uint8_t rv[3][kWin / 32];
  {
    const int base[3] = {i0 - kTubeS, win_base(j0, lj), win_base(k0, lk)};
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int h = 0; h < kWin / 32; ++h) {
        const int x = base[q] + lane + 32 * h;
        rv[q][h] = (x >= 0 && x < len[q]) ? (uint8_t)S[q][x] : (uint8_t)255;
      }
  }
  constexpr int V = (W + 3) / 4;  // 16-byte vectors per record (W = 2 uses the low half)
  uint4 v[kTubePer][V];
  bool valid[kTubePer];
#pragma unroll
  for (int u = 0; u < kTubePer; ++u) {
    const int e = lane + 32 * u;
    const int sx = e / (kTubeR * kTubeC), rem = e % (kTubeR * kTubeC);
    const int ii = i0 - sx;
    const int gr = ((j0 - sx) >> lj) + rem / kTubeC - 1;
    const int gc = ((k0 - sx) >> lk) + rem % kTubeC - 1;
    valid[u] = e < kTubeRecs && ii >= i_lo && gr >= 0 && gc >= 0 && gr < nJR && gc < nKC;
    if (valid[u]) {
      const int task = (gr / kPR) * nK + (gc / kPC);
      const int lr = gr % kPR, lcc = gc % kPC;
      const uint32_t* src =
          codes + (((int64_t)task * T + (ii - i_lo + lr + lcc)) * 32 + (lr * kPC + lcc)) * W;
      if (W == 2) {
        const uint2 h = __ldcg(reinterpret_cast<const uint2*>(src));
        v[u][0] = make_uint4(h.x, h.y, 0u, 0u);
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) v[u][q] = __ldcg(reinterpret_cast<const uint4*>(src) + q);
      }
    }
  }
  // All loads above are issued before any store below (the barrier keeps the compiler from
  // pairing each load with its store, which would serialise the round trips).
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int h = 0; h < kWin / 32; ++h) res[q][lane + 32 * h] = rv[q][h];
#pragma unroll
  for (int u = 0; u < kTubePer; ++u) {
    if (!valid[u]) continue;
    uint32_t* dst = win + (lane + 32 * u) * W;
    if (W == 2) {
      *reinterpret_cast<uint2*>(dst) = make_uint2(v[u][0].x, v[u][0].y);
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) reinterpret_cast<uint4*>(dst)[q] = v[u][q];
    }
  }
}

template <int W>
__global__ void __launch_bounds__(32) walk_kernel(const WalkParams p) {
  __shared__ uint4 win4[kTubeRecs * W / 4 + 1];
  __shared__ uint8_t res[3][kWin];
  uint32_t* win = reinterpret_cast<uint32_t*>(win4);
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x;
  const TripDesc& d = p.desc[p.tb_trips[q]];
  const int a = d.len[0], b = d.len[1], c = d.len[2];
  const int len[3] = {a, b, c};
  const int nK = d.nK, nJR = d.nJ * kPR, nKC = d.nK * kPC;
  const int lj = __ffs(p.NJ) - 1, lk = __ffs(p.NK) - 1;  // tile sides are powers of two
  const int8_t* const S[3] = {p.seq + d.s_off[0], p.seq + d.s_off[1], p.seq + d.s_off[2]};
  const int cap = p.row_cap[q];
  uint8_t* row0 = p.rows + p.row_off[q];
  uint8_t* row1 = row0 + cap;
  uint8_t* row2 = row1 + cap;
  const uint32_t* codes = p.codes + d.code_off;
  const int T = p.T_slab > 0 ? p.T_slab : d.T, i_lo = p.i_lo;
  const bool global = p.atype == kGlobal, local = p.atype == kLocal;
  int i = a, j = b, k = c, n = 0, bad = 0;
  if (p.state && !p.init_state) {  // a linear-space traceback resumes where the slab above left it
    i = p.state[4 * q];
    j = p.state[4 * q + 1];
    k = p.state[4 * q + 2];
    n = p.state[4 * q + 3];
  } else if (!global) {  // semi-global / local: the first cell with the best score
    const unsigned long long key = p.best64[d.out_idx];
    const unsigned long long lin = ((1ull << 37) - 1) - (key & ((1ull << 37) - 1));
    const unsigned long long bc = (unsigned long long)(b + 1) * (unsigned long long)(c + 1);
    i = (int)(lin / bc);
    j = (int)((lin % bc) / (unsigned long long)(c + 1));
    k = (int)(lin % (unsigned long long)(c + 1));
    if (lane == 0) p.scores[d.out_idx] = (int)(key >> 37) - (1 << 26);
    if (key == 0 || i > a || j > b || k > c) bad = 1;
  }
  const int ei = i, ej = j, ek = k;  // end cell of the alignment (for the span)
  // start cells: the origin (global), any axis cell (semi-global, local)
  const auto start = [&](int ii, int jj, int kk) {
    return global ? (ii | jj | kk) == 0 : (ii == 0) + (jj == 0) + (kk == 0) >= 2;
  };
  int done = start(i, j, k);
  while (!done && i >= i_lo && !bad) {
    const int i0 = i, j0 = j, k0 = k;
    tube_load<W>(win, res, i0, j0, k0, lj, lk, codes, len, nK, nJR, nKC, S, T, i_lo, lane);
    __syncwarp();
    // residue windows: S0[x - 1] is res[0][x - iw], and likewise for S1 and S2
    const int iw = i0 - kTubeS + 1, jw = win_base(j0, lj) + 1, kw = win_base(k0, lk) + 1;
    // rank of the move stored at cell (ci, cj, ck) if the tube holds it, else -1
    const auto rank_at = [&](int ci, int cj, int ck) -> int {
      const int sx = i0 - ci;
      if (sx >= kTubeS || ci < i_lo || cj < 0 || ck < 0) return -1;
      const int dr = (cj >> lj) - ((j0 - sx) >> lj) + 1;
      const int dc = (ck >> lk) - ((k0 - sx) >> lk) + 1;
      if ((unsigned)dr >= (unsigned)kTubeR || (unsigned)dc >= (unsigned)kTubeC) return -1;
      const int e = ((cj & ((1 << lj) - 1)) << lk) + (ck & ((1 << lk) - 1));
      const uint32_t word = win[((sx * kTubeR + dr) * kTubeC + dc) * W + (e >> 3)];
      return (word >> code_bit(e)) & 7;
    };
    for (;;) {  // warp-uniform
      // Lane m probes the cell m diagonal moves ahead; the run is the leading lanes whose cell
      // holds the (1,1,1) move (rank 7) and is no start cell.
      const int ci = i - lane, cj = j - lane, ck = k - lane;
      const int rk = rank_at(ci, cj, ck);
      const bool diag = rk == 7 && ci >= 1 && cj >= 1 && ck >= 1 && !start(ci, cj, ck);
      const unsigned nd = ~__ballot_sync(kFull, diag);
      const int run = nd ? __ffs(nd) - 1 : 32;
      if (run > cap - n) {  // longer than the rows: corrupt codes
        bad = 1;
        break;
      }
      if (lane < run) {
        const int pos = cap - 1 - (n + lane);
        row0[pos] = res[0][ci - iw];
        row1[pos] = res[1][cj - jw];
        row2[pos] = res[2][ck - kw];
      }
      i -= run;
      j -= run;
      k -= run;
      n += run;
      if (start(i, j, k)) {
        done = 1;
        break;
      }
      if (run == 32) continue;
      // The cell after the run: outside the tube (stage the next one), or a single other move.
      const int rank = __shfl_sync(kFull, rk, run);
      if (rank < 0) break;
      if (rank == 0 && local) {  // v = 0 won: the local alignment starts here
        done = 1;
        break;
      }
      // rank -> move (Eq. 1 listing order, rank 7 first)
      const int di = (0xE8 >> rank) & 1, dj = (0xD4 >> rank) & 1, dk = (0xB2 >> rank) & 1;
      if (rank == 0 || n >= cap || i < di || j < dj || k < dk) {
        bad = 1;
        break;
      }
      if (lane == 0) {
        const int pos = cap - 1 - n;
        row0[pos] = di ? res[0][i - iw] : (uint8_t)255;
        row1[pos] = dj ? res[1][j - jw] : (uint8_t)255;
        row2[pos] = dk ? res[2][k - kw] : (uint8_t)255;
      }
      i -= di;
      j -= dj;
      k -= dk;
      ++n;
      if (start(i, j, k)) {
        done = 1;
        break;
      }
    }
    __syncwarp();  // the next tube overwrites the shared buffers
  }
  if (lane == 0) {
    if (p.state) {
      p.state[4 * q] = i;
      p.state[4 * q + 1] = j;
      p.state[4 * q + 2] = k;
      p.state[4 * q + 3] = n;
    }
    if (bad) {
      atomicOr(p.err, 2);
      p.aln_len[q] = -1;
    } else if (done) {
      p.aln_len[q] = n;
      if (p.span) {
        int* sp = p.span + 6 * q;
        sp[0] = i;
        sp[1] = j;
        sp[2] = k;
        sp[3] = p.state ? a : ei;  // a slab walk ends at (a, b, c)
        sp[4] = p.state ? b : ej;
        sp[5] = p.state ? c : ek;
      }
    }
  }
}

namespace {

template <int NJ, int NK, bool TB>
const void* kptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, TB, kGlobal, 0, false>);
}

const void* pick(int nj, int nk, bool tb, int at, int pk, bool slab) {
  if (slab) return (pk || at != kGlobal) ? nullptr : wavefront_slab(nj, nk, tb);
  if (pk >= 3) return tb ? nullptr : wavefront_vl(nj, nk, pk - 3, at);
  if (pk) return (tb || at != kGlobal) ? nullptr : wavefront_packed(nj, nk, pk);
  if (at != kGlobal) return wavefront_variant(nj, nk, at, tb);
  if (nj == 8 && nk == 8) return tb ? kptr<8, 8, true>() : kptr<8, 8, false>();
  if (nj == 4 && nk == 8) return tb ? kptr<4, 8, true>() : kptr<4, 8, false>();
  if (nj == 4 && nk == 4) return tb ? kptr<4, 4, true>() : kptr<4, 4, false>();
  // 8x4 (32 x 32-cell tasks) for traceback keys only: single triplets whose time is the ramp
  // cross fewer k-levels, whose lag is the larger one (8 lane columns of skew)
  if (nj == 8 && nk == 4) return tb ? kptr<8, 4, true>() : nullptr;
  return nullptr;
}

}  // namespace

int wavefront_block_threads(int pk) { return 32 * (pk >= 3 ? wavefront_vl_warps(pk - 3) : kWarpsPerCta); }

size_t wavefront_smem_bytes(int nj, int nk, int KP, bool pk) {
  const int WJ = kPR * nj, WK = kPC * nk;
  const int slot = kPC * (nk + 4) + WJ;
  const size_t sigN = (size_t)((KP * KP + 3) & ~3);
  const size_t nprof = pk ? 2 : 1;  // packed mode: a profile set per half
  return (sigN + (size_t)kWarpsPerCta * (nprof * KP * ((WJ + 4) + (WK + 4)) + kRing * slot)) *
         sizeof(int);
}

int wavefront_occupancy(int nj, int nk, bool tb, int at, int pk, bool slab, size_t smem,
                        int* blocks_per_sm) {
  const void* k = pick(nj, nk, tb, at, pk, slab);
  if (!k) return -1;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return -2;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, wavefront_block_threads(pk),
                                                    smem) != cudaSuccess)
    return -2;
  return 0;
}

int launch_wavefront(int nj, int nk, bool tb, int at, int pk, bool slab, const WaveParams& p,
                     int grid, size_t smem, void* stream) {
  const void* k = pick(nj, nk, tb, at, pk, slab);
  if (!k) return -1;
  void* args[] = {const_cast<WaveParams*>(&p)};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(wavefront_block_threads(pk)), args,
                                         smem, (cudaStream_t)stream);
  return e == cudaSuccess ? 0 : -2;
}

int launch_walk(const WalkParams& p, void* stream) {
  if (p.ntb <= 0) return 0;
  const int W = p.NJ * p.NK / 8;
  cudaStream_t st = (cudaStream_t)stream;
  if (W == 2) walk_kernel<2><<<p.ntb, 32, 0, st>>>(p);
  else if (W == 4) walk_kernel<4><<<p.ntb, 32, 0, st>>>(p);
  else if (W == 8) walk_kernel<8><<<p.ntb, 32, 0, st>>>(p);
  else return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace trioseq

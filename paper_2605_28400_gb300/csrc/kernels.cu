// kernels.cu — sm_103a kernels of the 3-way alignment engine: the global-alignment
// instantiations of the wavefront kernel (wavefront.cuh), the traceback walk, and the launchers.
//
// walk_kernel: one warp per traceback request. Lane 0 follows the stored moves back from
//   (a, b, c) through a tube of code records along the diagonal, staged in shared memory by the
//   whole warp in one round trip; repeated until the origin. In the linear-space traceback the
//   codes hold one slab of slices at a time: the walk resumes from a saved (i, j, k, n) and stops
//   when it leaves the slab.
#include "wavefront.cuh"

namespace trioseq {
// ---------------------------------------------------------------------------------------------
// Traceback walk. Optimal paths of related sequences run close to the cube's main diagonal, so
// the warp stages a "tube" of code records along the diagonal from the current cell: for each
// of the next kTubeS slices, the 3 x 3 lane tiles around the diagonal cell. All lanes load the
// tube in one round trip (independent loads, then shared-memory stores); lane 0 then follows
// the stored moves until the path leaves the tube, and the warp stages the next tube there.
constexpr int kTubeS = 32, kTubeR = 3, kTubeC = 3;
constexpr int kTubeRecs = kTubeS * kTubeR * kTubeC;
constexpr int kTubePer = (kTubeRecs + 31) / 32;

template <int W>
__device__ __forceinline__ void tube_load(uint32_t* win, int i0, int j0, int k0, int lj, int lk,
                                          const uint32_t* codes, const TripDesc& d, int T,
                                          int i_lo, int lane) {
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
    valid[u] = e < kTubeRecs && ii >= i_lo && gr >= 0 && gc >= 0 && gr < d.nJ * kPR &&
               gc < d.nK * kPC;
    if (valid[u]) {
      const int task = (gr / kPR) * d.nK + (gc / kPC);
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
  uint32_t* win = reinterpret_cast<uint32_t*>(win4);
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x;
  const TripDesc& d = p.desc[p.tb_trips[q]];
  const int a = d.len[0], b = d.len[1], c = d.len[2];
  const int lj = __ffs(p.NJ) - 1, lk = __ffs(p.NK) - 1;  // tile sides are powers of two
  const int8_t* S0 = p.seq + d.s_off[0];
  const int8_t* S1 = p.seq + d.s_off[1];
  const int8_t* S2 = p.seq + d.s_off[2];
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
    tube_load<W>(win, i0, j0, k0, lj, lk, codes, d, T, i_lo, lane);
    __syncwarp();
    if (lane == 0) {
      while (!done && i >= i_lo) {
        const int sx = i0 - i;
        if (sx >= kTubeS) break;
        const int dr = (j >> lj) - ((j0 - sx) >> lj) + 1;
        const int dc = (k >> lk) - ((k0 - sx) >> lk) + 1;
        if ((unsigned)dr >= (unsigned)kTubeR || (unsigned)dc >= (unsigned)kTubeC) break;
        const int e = ((j & ((1 << lj) - 1)) << lk) + (k & ((1 << lk) - 1));
        const uint32_t word = win[((sx * kTubeR + dr) * kTubeC + dc) * W + (e >> 3)];
        const int rank = (word >> code_bit(e)) & 7;
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
        const int pos = cap - 1 - n;
        row0[pos] = di ? (uint8_t)S0[i - 1] : (uint8_t)255;
        row1[pos] = dj ? (uint8_t)S1[j - 1] : (uint8_t)255;
        row2[pos] = dk ? (uint8_t)S2[k - 1] : (uint8_t)255;
        i -= di;
        j -= dj;
        k -= dk;
        ++n;
        done = start(i, j, k);
      }
    }
    __syncwarp();
    i = __shfl_sync(kFull, i, 0);
    j = __shfl_sync(kFull, j, 0);
    k = __shfl_sync(kFull, k, 0);
    n = __shfl_sync(kFull, n, 0);
    bad = __shfl_sync(kFull, bad, 0);
    done = __shfl_sync(kFull, done, 0);
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
  if (pk) return (tb || at != kGlobal) ? nullptr : wavefront_packed(nj, nk, pk);
  if (at != kGlobal) return wavefront_variant(nj, nk, at, tb);
  if (nj == 8 && nk == 8) return tb ? kptr<8, 8, true>() : kptr<8, 8, false>();
  if (nj == 4 && nk == 8) return tb ? kptr<4, 8, true>() : kptr<4, 8, false>();
  if (nj == 4 && nk == 4) return tb ? kptr<4, 4, true>() : kptr<4, 4, false>();
  return nullptr;
}

}  // namespace

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
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kWarpsPerCta * 32, smem) !=
      cudaSuccess)
    return -2;
  return 0;
}

int launch_wavefront(int nj, int nk, bool tb, int at, int pk, bool slab, const WaveParams& p,
                     int grid, size_t smem, void* stream) {
  const void* k = pick(nj, nk, tb, at, pk, slab);
  if (!k) return -1;
  void* args[] = {const_cast<WaveParams*>(&p)};
  const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kWarpsPerCta * 32), args, smem,
                                         (cudaStream_t)stream);
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

// engine.h — data layouts shared by the host runtime and the CUDA kernels.
//
// Frame and encoding used on the device (all exact integer transforms of Eq. 1):
//  * Potential shift. Every move adds 2*alpha per residue it consumes on top of the pairwise
//    terms, so with M'[i][j][k] = M[i][j][k] - 2*alpha*(i+j+k) the single-residue moves cost 0,
//    a two-residue move costs sigma''(x,y) and the three-residue move costs
//    sigma''(x,y) + sigma''(x,z) + sigma''(y,z), where sigma'' = sigma - 2*alpha.
//    The score is M'[a][b][c] + 2*alpha*(a+b+c).
//  * Virtual residue. Each sequence gets a virtual residue VIRT = K at position 0 and the cube
//    is indexed 0..a, 0..b, 0..c directly; sigma''(VIRT, .) = 0. Cells at index -1 are -infinity
//    (kNeg) except M'[-1][-1][-1] = 0, so the ordinary 7-move recurrence reproduces M_000 = 0,
//    the axis values and the face recurrences of Sec. II without special cases.
//  * Traceback keys. With traceback, a cell stores 8*M' + 7; every candidate adds 8*cost plus
//    (rank - 7), rank 7..1 following Eq. 1's listing order. One integer max then yields the
//    score and the winning move of the tie-break; the low 3 bits of the max are the rank.
#pragma once
#include <stdint.h>

namespace trioseq {

constexpr int kNeg = -(1 << 30);   // -infinity sentinel (never accumulates: see the kernel)
// A boundary-record slot not yet written (the byte 0x80 repeated): below -infinity and below any
// key, so no stored value can equal it.
constexpr int kRecordSentinel = (int)0x80808080u;
constexpr int kPR = 4;             // lanes of a warp along j
constexpr int kPC = 8;             // lanes of a warp along k
constexpr int kMaxAlphabet = 32;
constexpr int kWarpsPerCta = 4;
constexpr int kRing = 4;           // face-staging ring slots per warp (power of two)

// Alignment types of Sec. II. Semi-global: zero axes, score = best cell on a last slice;
// local: zero axes and v = 0 in Eq. 1, score = best cell. Both are score-only on the device.
constexpr int kGlobal = 0, kSemiGlobal = 1, kLocal = 2;

// Packed int16x2 mode (global score only): two triplets share a column task, one per 16-bit half
// of every register, record word and halo. -infinity is kNeg16 in each half. A batch is packed
// only if every cell value of both halves stays within +-(2^14 - 3*max|sigma''|), so no add wraps
// and the sentinel never wins against a finite candidate.
constexpr int kNeg16 = -(1 << 14);
constexpr int kNeg16x2 = (int)0xC000C000u;  // kNeg16 in both halves
// Biased packed mode (all sigma'' >= 0): a half stores M' + 2^14; -infinity is 0, M' = 0 is
// kBias16x2. Real M' are >= 0 there, so real halves are >= 2^14 and every sum stays below 2^16.
constexpr int kBias16x2 = 0x40004000;

// Rank of each move in the tie-break (Eq. 1 listing order): rank 7 wins ties over rank 6 ...
// rank -> (di, dj, dk):
//   7:(1,1,1) 6:(1,1,0) 5:(1,0,1) 4:(0,1,1) 3:(1,0,0) 2:(0,1,0) 1:(0,0,1)
//
// Traceback code layout. Lane (r, lc) of column task (J, K) writes, at step t (slice
// i = t - r - lc), one record of NJ*NK/8 32-bit words at word offset
//   code_off + ((task * T + t) * 32 + lane) * (NJ*NK/8),   task = J*nK + K, lane = r*8 + lc.
// Cell (p, q) of the lane tile is e = p*NK + q; it lives in word e/8 at bit
//   8*(e & 3) + 4*((e >> 2) & 1)   (the 3-bit rank in the low bits of that nibble).
__host__ __device__ inline int code_bit(int e) { return 8 * (e & 3) + 4 * ((e >> 2) & 1); }

// Face records. Column task (J, K) publishes, per slice s (0..a):
//   its last j-row in the j-record  Oj[s][0 .. WK+3]: slot 3 = M'[s][J*WJ+WJ-1][K*WK-1] (the
//     corner its consumer needs), slots 4 .. WK+3 = M'[s][J*WJ+WJ-1][K*WK + kl];
//   its last k-column in the k-record Ok[s][0 .. WJ-1] = M'[s][J*WJ + jl][K*WK+WK-1].
// Records of one task are contiguous: Oj at oj_off + task*(a+1)*(WK+4), Ok at
// ok_off + task*(a+1)*WJ (int32 offsets into the face workspace).

struct TripDesc {
  int64_t s_off[3];    // byte offsets of S0, S1, S2 in the packed residue buffer
  int64_t oj_off;      // int32 offset of this triplet's j-records in the face workspace
  int64_t ok_off;      // int32 offset of its k-records
  int64_t code_off;    // uint32-word offset of its traceback codes (-1: score only)
  int64_t prog_base;   // index of task (J=0,K=0) in the progress array
  int32_t len[3];      // a, b, c
  int32_t glen[3];     // lengths of the task grid: len, or in packed mode the pair's maxima
  int32_t pair;        // packed mode: descriptor of the triplet in the high halves; else -1
  int32_t nJ, nK;      // column blocks along j and k
  int32_t T;           // steps per column task: a + 1 + (kPR - 1) + (kPC - 1)
  int32_t score_base;  // 2*alpha*(a+b+c)
  int32_t out_idx;     // index into the score output
  int32_t tb_idx;      // index among the batch's traceback triplets (-1: none)
};

struct Task {
  int32_t trip, J, K, pad;
};

struct WaveParams {
  const TripDesc* desc;
  const Task* tasks;
  int32_t ntasks;
  int32_t KP;          // alphabet size + 1 (virtual residue)
  const int8_t* seq;   // packed residue codes
  const int32_t* sig;  // KP*KP table of sigma'' (x8 in traceback mode), VIRT row/col = 0
  int32_t* faces;
  int32_t* progress;   // one published step count per task, zeroed before launch
  int32_t* queue;      // work-queue head, zeroed before launch
  uint32_t* codes;     // packed 4-bit traceback codes (traceback mode)
  int32_t* scores;     // per-triplet output
  int32_t* err;        // device error word (bit 0: a bounded wait expired)
  int32_t TI;          // publish progress every TI steps
  int64_t wait_ns;     // a wait that sees no progress for this long gives up
  int32_t g2;          // -2*alpha (>= 0): the potential shift per consumed residue
  // Slab launches (one triplet, global type, int32): the launch covers the slices
  // i0 .. i0 + desc.len[0] of the cube. plane_in holds the stored values of slice i0 - 1 (null:
  // i0 = 0, the cube's own start); plane_out, if set, receives the slab's last slice. Planes
  // span the padded task grid: (nJ*WJ) rows of (nK*WK) int32, row-major in (j, k).
  int32_t i0;
  const int32_t* plane_in;
  int32_t* plane_out;
  // Semi-global / local with traceback: per triplet, the 64-bit max of
  // (M + 2^26) << 37 | (2^37 - 1 - cell index), i.e. the best score and its first cell in
  // (i, j, k) order; zeroed before launch. The walk starts there and writes the score.
  unsigned long long* best64;
  // First-wave pacing (launches of at least two waves of tasks): queue task n < pace_n starts
  // once task 0 (no producers, never waits) has published n * pace_T / pace_n steps at
  // *pace_flag, spreading the first wave's starts, hence its completions, over one task
  // duration; 0 disables.
  int32_t pace_n, pace_T;
  const int32_t* pace_flag;
  int32_t one;         // 1, as a launch argument (multiply-adds by it stay on the FMA pipe)
  // Traceback launches: the boundary records start as kRecordSentinel (set before the launch)
  // and a consumer waits on the record slots themselves instead of the producers' progress.
  int32_t data_flags;
};

struct WalkParams {
  const TripDesc* desc;
  const int32_t* tb_trips;   // triplet index of each traceback request
  int32_t ntb;
  const int8_t* seq;
  const uint32_t* codes;
  uint8_t* rows;             // per request: 3 rows of cap bytes, residue codes, 255 = gap
  const int64_t* row_off;    // byte offset of each request's rows
  const int32_t* row_cap;    // capacity (a+b+c) of each row
  int32_t* aln_len;          // written: alignment length (the alignment is the last L bytes)
  int32_t* err;              // bit 1: corrupt code met during a walk
  int32_t NJ, NK;            // tile of the wavefront variant that wrote the codes
  // Slab walks (linear-space traceback): codes hold only the slices i_lo .. of a slab launch
  // with T_slab steps per task; state (i, j, k, n per request) carries the walk across slabs.
  // i_lo = 0, T_slab = 0 and state = null walk the whole cube from (a, b, c) in one launch.
  int32_t i_lo, T_slab;
  int32_t* state;
  int32_t init_state;        // 1: start at (a, b, c) (the top slab) instead of reading state
  int32_t atype;             // alignment type: semi-global and local start at best64's cell,
  const unsigned long long* best64;  // stop at axis cells, and local also at rank 0 (v won)
  int32_t* scores;           // written from best64 for those types
  int32_t* span;             // per request: begin (i, j, k) and end (i, j, k) of the alignment
};

// Affine gaps (affine.cu): natural gap costs, 13 reachable states per cell, score only.
constexpr int kAffineStates = 13;
struct AffineParams {
  const TripDesc* desc;
  const Task* tasks;      // queue: one entry per triplet (Task.trip), largest cube first
  int32_t n;
  int32_t KP;
  const int8_t* seq;
  const int32_t* sub;     // KP x KP table of sigma (the virtual row and column unused)
  int32_t gap, gap_open;  // alpha (per residue against a gap), gamma (per maximal gap run)
  int32_t* planes;        // per CTA: 4 plane buffers of plane_cells * 16 int32 (13 used)
  int64_t plane_cells;    // (max b + 1) * (max c + 1) over the batch
  int32_t* queue;         // zeroed before launch
  int32_t* scores;
};
int affine_occupancy(int* blocks_per_sm);
int launch_affine(const AffineParams& p, int grid, void* stream);

// Host-side launchers implemented in kernels.cu. `at` is the alignment type (kGlobal, ...);
// semi-global and local exist for score mode (tb = false) only, and their scores are
// accumulated with atomicMax, so the score array must hold INT_MIN-like values before launch.
// `slab` selects the slab-launch instantiations (global type, int32, either mode).
// `pk` is the packed mode: 0 int32, 1 signed int16x2, 2 biased unsigned int16x2, 3 two cells of
// one triplet per register, 4 and 5 the same with the sigma''(y,z) tile in shared memory (2-warp
// and 1-warp CTAs).
int launch_wavefront(int nj, int nk, bool tb, int at, int pk, bool slab, const WaveParams& p,
                     int grid, size_t smem, void* stream);
int wavefront_occupancy(int nj, int nk, bool tb, int at, int pk, bool slab, size_t smem,
                        int* blocks_per_sm);
// Kernel entry of a semi-global or local instantiation (kernels_variants.cu), or null.
const void* wavefront_variant(int nj, int nk, int at, bool tb);
// Kernel entry of a packed int16x2 (global, score) instantiation (kernels_packed.cu), or null.
const void* wavefront_packed(int nj, int nk, int mode);
// two cells of one triplet per register (wavefront_vl.cuh): nj x nk = 8 x 16 or 8 x 8 cells per
// lane; cs = 1 or 2: the lane's sigma''(y,z) tile in shared memory (8 x 16 only; 2-warp or
// 1-warp CTAs), 0: in registers
const void* wavefront_vl(int nj, int nk, int cs, int at);
size_t wavefront_vl_smem_bytes(int nj, int nk, int KP, int cs);
int wavefront_vl_warps(int cs);
// Kernel entry of a slab-launch instantiation (kernels_slab.cu), or null.
const void* wavefront_slab(int nj, int nk, bool tb);
int launch_walk(const WalkParams& p, void* stream);
size_t wavefront_smem_bytes(int nj, int nk, int KP, bool pk);
// threads per CTA of a launch in packed mode pk (2 warps for pk = 4, 1 for pk = 5, else
// kWarpsPerCta)
int wavefront_block_threads(int pk);

}  // namespace trioseq

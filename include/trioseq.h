/*
 * trioseq.h — C ABI of the GB300 engine for exact 3-way global sequence alignment.
 *
 * The operation (Graca & Ilic, "TrioSeq", Sec. II): three sequences S0, S1, S2 of lengths
 * a, b, c over an alphabet, a symmetric substitution score sigma and a linear gap alpha are
 * aligned by the dynamic program of Eq. 1 over the (a+1) x (b+1) x (c+1) cube:
 *
 *   M[i][j][k] = max over the 7 moves m = (di,dj,dk) in {0,1}^3 \ {(0,0,0)} of
 *                M[i-di][j-dj][k-dk] + SOP(column emitted by m),
 *   SOP(x,y,z) = sigma(x,y) + sigma(x,z) + sigma(y,z),
 *
 * where a column holds the residue S0[i-1] if di = 1 and a gap otherwise (likewise for S1, S2),
 * sigma(residue, gap) = alpha and sigma(gap, gap) = 0 (Sec. II, SOP definition). Global alignment
 * (Sec. II, "Global Alignments"): M[0][0][0] = 0, predecessors outside the cube are -infinity,
 * and the optimal score is M[a][b][c]. The optimal alignment is recovered by walking the winning
 * moves back from (a,b,c) to the origin.
 *
 * Tie-break (the paper leaves it open): when several moves reach the maximum, the first one in
 * Eq. 1's listing order wins: (1,1,1) > (1,1,0) > (1,0,1) > (0,1,1) > (1,0,0) > (0,1,0) > (0,0,1).
 * With it the emitted alignment is unique, so results are reproducible bit for bit.
 *
 * Conventions for every call:
 *  - Every call returns a trioseq_status and never aborts the process: no C++ exception crosses
 *    the C boundary, and a failed host allocation returns TRIOSEQ_ENOMEM. For tests, setting
 *    TRIOSEQ_TEST_HOST_BAD_ALLOC=1 in the environment before the first call makes every call
 *    except trioseq_strerror fail that way, before it touches its arguments or the GPU.
 *  - The caller owns all inputs and outputs; the library copies what it needs before returning
 *    (host inputs) or reads device inputs only inside the call's stream order.
 *  - Handles are opaque and released by the matching *_destroy call.
 *  - Scores are int32. A call whose worst-case score bound does not fit the engine's integer range
 *    (|score| * 8 must stay below 2^29, see trioseq_plan) fails with TRIOSEQ_EOVERFLOW.
 *  - A handle may be used by one host thread at a time; the server (trioseq_server_*) is the
 *    thread-safe entry for concurrent producers.
 *  - The compute path is CUDA only (sm_103a). Without a usable GPU the calls fail with
 *    TRIOSEQ_ECUDA; there is no CPU fallback.
 */
#ifndef TRIOSEQ_H
#define TRIOSEQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TRIOSEQ_OK = 0,
  TRIOSEQ_EINVAL = 1,    /* bad argument: null pointer, residue outside the alphabet,
                            asymmetric sigma, gap > 0, cap too small, unknown index */
  TRIOSEQ_ENOMEM = 2,    /* host or device allocation failed */
  TRIOSEQ_EAGAIN = 3,    /* result not ready yet (poll) or server queue full (submit) */
  TRIOSEQ_EOVERFLOW = 4, /* score bound exceeds the integer range of the engine */
  TRIOSEQ_ETIMEOUT = 5,  /* a bounded device-side wait expired; the context stays usable */
  TRIOSEQ_ECUDA = 6,     /* CUDA runtime error or no usable GPU */
  TRIOSEQ_ENOTIMPL = 7,  /* requested feature is not built */
  TRIOSEQ_ESCRATCH = 8   /* request needs more than the fixed scratch of trioseq_align_noalloc */
} trioseq_status;

/* Scoring scheme (Sec. II). `alphabet` lists the residue characters (1..32 distinct bytes);
 * `sub` is the alphabet_size x alphabet_size row-major substitution matrix, which must be
 * symmetric; `gap` is alpha, added once per residue-gap pair in a column (so a column with one
 * residue and two gaps scores 2*alpha), and must be <= 0. */
typedef struct {
  const char* alphabet;
  int32_t alphabet_size;
  const int8_t* sub;
  int32_t gap;
} trioseq_scoring;

/* One triplet: three caller-owned host strings over the plan's alphabet (not NUL-terminated;
 * lengths given explicitly, 0 allowed). */
typedef struct {
  const char* s[3];
  uint32_t len[3];
} trioseq_triplet;

enum { TRIOSEQ_SCORE_ONLY = 0, TRIOSEQ_WITH_TRACEBACK = 1 };

/* Alignment types of Sec. II, given to trioseq_plan as `flags`:
 *  GLOBAL      M[0][0][0] = 0, v = -infinity, score = M[a][b][c] ("Global Alignments").
 *  SEMIGLOBAL  the axes are zero, M[i][0][0] = M[0][j][0] = M[0][0][k] = 0, v = -infinity; the
 *              score is the best cell on a last slice, max of M over i = a or j = b or k = c
 *              ("Semi-Global Alignments"). Only the axes are zero-initialised (the faces follow
 *              Eq. 1), as the section writes it.
 *  LOCAL       the same zero axes and v = 0 in Eq. 1 (no cell is negative); the score is the
 *              best cell of the cube ("Local Alignments").
 * With WITH_TRACEBACK, SEMIGLOBAL and LOCAL report the alignment of the best cell: the first cell
 * in (i, j, k) order holding the best score among the cells that count. The walk back from it
 * takes the first maximal candidate in Eq. 1's order, v listed last, and stops at an axis cell
 * (two zero indices) or, for LOCAL, where v = 0 alone is maximal. The rows are that path's
 * columns. trioseq_traceback_span gives the cells it joins, i.e. the substrings it aligns.
 * Such batches need (a+1)(b+1)(c+1) < 2^37 per triplet (else EOVERFLOW). */
enum { TRIOSEQ_GLOBAL = 0, TRIOSEQ_SEMIGLOBAL = 1, TRIOSEQ_LOCAL = 2 };

typedef struct trioseq_plan_s* trioseq_plan_t;

/* trioseq_plan — validate a scoring scheme and create a plan.
 * The plan owns the device workspace (grown on demand), the kernel-variant choice and the
 * autotuner cache for the current CUDA device. `max_len_hint` pre-sizes nothing mandatory
 * (0 = no hint). `flags` is the alignment type: TRIOSEQ_GLOBAL (0), TRIOSEQ_SEMIGLOBAL or
 * TRIOSEQ_LOCAL; every call on the plan (batches, autotuner, server) uses that type.
 * Tuning read from the environment when the plan is created (none changes a result):
 * TRIOSEQ_SCORE_TILE forces the score tile ("8x8", "4x8", "4x4", or the two-cells-per-register
 * "8x16", "8x8v", "8x16s", "8x16t"; work those cannot take runs on the int32 8x8 kernel) and
 * TRIOSEQ_TB_TILE the traceback tile ("8x8", "4x8", "4x4", "8x4"); TRIOSEQ_TI the progress
 * interval (steps between published progress counts, default 8); TRIOSEQ_DATA_FLAGS=1/0 forces
 * the boundary records to act as their own readiness flags in traceback launches, or not (by
 * default they do for one-triplet traceback batches); TRIOSEQ_PACKED=0 disables two triplets per
 * register; TRIOSEQ_GRAPHS=0 graph replay; TRIOSEQ_PACE=0 first-wave pacing; TRIOSEQ_WAIT_MS the
 * bounded waits' limit (default 2000). TRIOSEQ_CTAS_PER_SM (read per batch) caps the resident
 * CTAs per SM.
 * Errors: EINVAL (null, bad alphabet, asymmetric sub, gap > 0, unknown flags), ECUDA. */
trioseq_status trioseq_plan(const trioseq_scoring* scoring, uint32_t max_len_hint, uint32_t flags,
                            trioseq_plan_t* out);

/* trioseq_plan_affine — a plan for the sum-of-pairs score with affine gaps. The paper names
 * affine gaps as future work (Sec. VI) and gives no definition; this library reads them as
 * natural gap costs (Altschul 1989) in Gotoh's affine form: each pair's induced pairwise
 * alignment (the columns with a gap in both of its sequences deleted) scores sub[x][y] per
 * residue pair, scoring->gap (alpha) per residue against a gap, and gap_open (gamma) once per
 * maximal run of gaps in one of its sequences. gap_open = 0 gives the linear model of Sec. II.
 * Arguments: scoring as for trioseq_plan; gap_open <= 0 (>= -2^20); flags must be
 * TRIOSEQ_GLOBAL. The plan serves trioseq_align_batch and the device-resident batch calls in
 * score-only mode (traceback: ENOTIMPL); trioseq_plan_autotune has nothing to choose. The
 * kernel keeps 13 int32 states per cell and sweeps anti-diagonal planes (one CTA per triplet).
 * Errors: EINVAL (as trioseq_plan, gap_open out of range, other flags), ENOMEM, ECUDA;
 * EOVERFLOW at batch time when (3 max|sub| + 3|gap| + 3|gap_open|) * (a+b+c) >= 2^29. */
trioseq_status trioseq_plan_affine(const trioseq_scoring* scoring, int32_t gap_open,
                                   uint32_t flags, trioseq_plan_t* out);

/* Release a plan and its device memory. Null is accepted. Destroy the plan's device-resident
 * batches and any server that names it first. The call waits for the plan's own last
 * trioseq_align_batch work only; it synchronises no other stream (a running server's included),
 * and the memory is freed in the order of the plan's private stream. */
trioseq_status trioseq_plan_destroy(trioseq_plan_t plan);

/* trioseq_align_batch — align n triplets (host strings) in one persistent launch.
 * mode: TRIOSEQ_SCORE_ONLY or TRIOSEQ_WITH_TRACEBACK. scores_out: caller-owned host array of n
 * int32, filled before return. stream: a cudaStream_t (NULL = the legacy default stream); the
 * call synchronises that stream before returning.
 * With TRACEBACK the alignments stay in the plan until the next align call and are read with
 * trioseq_traceback.
 * Work: encode + pack (host), one H2D copy, one persistent wavefront launch over all triplets,
 * one traceback-walk launch (traceback mode), one D2H copy of scores (and alignments).
 * Errors: EINVAL (residue outside the alphabet, null), EOVERFLOW, ENOMEM, ETIMEOUT, ECUDA. */
trioseq_status trioseq_align_batch(trioseq_plan_t plan, const trioseq_triplet* triplets, size_t n,
                                   uint32_t mode, int32_t* scores_out, void* stream);

/* trioseq_traceback — copy the optimal alignment of triplet `idx` of the last TRACEBACK batch.
 * row0/row1/row2 receive the three aligned rows (alphabet characters, '-' for gaps, not
 * NUL-terminated); cap is the capacity of each row; *aln_len receives the length L
 * (max(a,b,c) <= L <= a+b+c). If cap < L the call returns EINVAL and still sets *aln_len.
 * Errors: EINVAL (no traceback batch, idx out of range, cap too small, null). */
trioseq_status trioseq_traceback(trioseq_plan_t plan, size_t idx, char* row0, char* row1,
                                 char* row2, size_t cap, size_t* aln_len);

/* trioseq_traceback_span — the cells the alignment of triplet idx joins: begin = (i0, j0, k0),
 * end = (i1, j1, k1); its rows align S0[i0:i1], S1[j0:j1], S2[k0:k1]. For GLOBAL plans begin =
 * (0,0,0) and end = (a,b,c); for SEMIGLOBAL begin lies on an axis and end on a last face.
 * Errors: EINVAL (no traceback batch, idx out of range, null). */
trioseq_status trioseq_traceback_span(trioseq_plan_t plan, size_t idx, int32_t begin[3],
                                      int32_t end[3]);

/* ---- device-resident batches (inputs already in HBM; used by benchmarks and servers) ---- */

typedef struct trioseq_batch_s* trioseq_batch_t;

/* trioseq_batch_create — encode, pack and upload n triplets once; build the work queue, the
 * triplet descriptors and the workspace layout. The batch can then be run repeatedly with
 * trioseq_batch_run without any host-to-device traffic. The plan must outlive the batch.
 * Errors: EINVAL, EOVERFLOW, ENOMEM, ECUDA. */
trioseq_status trioseq_batch_create(trioseq_plan_t plan, const trioseq_triplet* triplets,
                                    size_t n, uint32_t mode, trioseq_batch_t* out);

/* trioseq_batch_run — enqueue one full pass of the hot path on `stream` (workspace reset, the
 * persistent wavefront kernel, and the traceback walk in traceback mode). Asynchronous: scores
 * land in device memory; read them with trioseq_batch_scores. The pass is captured once into a
 * CUDA graph (on a private stream, so `stream` may be the legacy default stream) and every run
 * replays it with one graph launch; the graph is captured again when profiling is switched or
 * the batch's buffers moved. Setting the environment variable TRIOSEQ_GRAPHS=0 before
 * trioseq_plan makes the runs of that plan's batches plain launches instead.
 * Errors: ECUDA (capture, instantiation or launch failure). */
trioseq_status trioseq_batch_run(trioseq_batch_t batch, void* stream);

/* trioseq_batch_scores — synchronise `stream`, check the device error word, and copy the n
 * scores to the caller's host array. Errors: ETIMEOUT (bounded device wait expired), ECUDA. */
trioseq_status trioseq_batch_scores(trioseq_batch_t batch, void* stream, int32_t* scores_out);

/* Device address of the batch's int32 score array (n entries), valid until destroy. */
trioseq_status trioseq_batch_device_scores(trioseq_batch_t batch, int32_t** d_scores);

/* trioseq_batch_alignment — after trioseq_batch_scores in traceback mode: copy the alignment of
 * triplet idx as in trioseq_traceback. */
trioseq_status trioseq_batch_alignment(trioseq_batch_t batch, size_t idx, char* row0, char* row1,
                                       char* row2, size_t cap, size_t* aln_len);

/* trioseq_batch_span — as trioseq_traceback_span, for triplet idx of a device-resident batch. */
trioseq_status trioseq_batch_span(trioseq_batch_t batch, size_t idx, int32_t begin[3],
                                  int32_t end[3]);

/* Work statistics of a batch: number of triplets, the paper's cell count
 * (sum of |S0|*|S1|*|S2|, the TCUPS numerator), the number of column tasks in the queue, and the
 * kernel variant chosen (tile rows x tile cols per lane; the two-cells-per-register tiles count
 * both halves, so 8x8v reads 8 x 8, told apart from the int32 8x8 by trioseq_batch_packing).
 * Any out pointer may be null. */
trioseq_status trioseq_batch_info(trioseq_batch_t batch, size_t* n, uint64_t* cells,
                                  uint64_t* tasks, int32_t* tile_j, int32_t* tile_k);

/* trioseq_batch_packing — *per_word = how many DP cells share each register of the batch's
 * kernel: 2 in the packed int16x2 modes, else 1. Two packed modes are the integer counterpart
 * of the paper's FP16x2 arithmetic (Sec. IV-B): two triplets per register, or two column halves
 * of one triplet per register (a one-triplet batch whose score tile is 8x16 or "8x8v", see
 * trioseq_plan_autotune). A score-only global batch of two or more triplets
 * is packed when every pair fits: the batch pairs triplets of the same column-task grid class,
 * and each pair's grid needs max|sigma''| * (a+b+c+3) < 2^14 on its maximal lengths. Otherwise,
 * or with TRIOSEQ_PACKED=0 set before trioseq_plan, every triplet gets its own int32 tasks.
 * Results are identical either way. Errors: EINVAL (null). */
trioseq_status trioseq_batch_packing(trioseq_batch_t batch, int32_t* per_word);

/* trioseq_batch_kernel — the wavefront kernel a batch launches, as a NUL-terminated name with
 * its template arguments and tile label (for example "wavefront_vl_kernel<8,4,false> tile 8x8v",
 * "wavefront_vl_kernel<8,8,true> tile 8x16s" or "wavefront_kernel<8,4,traceback,global> tile
 * 8x4"), written into name[0..cap). The "8x16s" tile keeps the lane's sigma''(y,z) tile and
 * 16-bit profiles in shared memory and runs 2-warp CTAs. Errors: EINVAL (null, cap too small:
 * the name is then cut). */
trioseq_status trioseq_batch_kernel(trioseq_batch_t batch, char* name, size_t cap);

/* trioseq_batch_slabs — slab layout of a one-triplet batch: *slices = slices per slab, *slabs =
 * number of slabs, both 0 when the cube runs in one launch.
 * A one-triplet, global-type batch runs in slabs when its boundary records, plus with traceback
 * its 4-bit codes, would exceed the plan's budget at once. The budget is half the free device
 * memory at trioseq_plan, or TRIOSEQ_SLAB_BUDGET_MB; TRIOSEQ_SLAB_SLICES forces a slab height.
 * Each slab launch starts from the plane of stored values its predecessor left. Score mode
 * keeps two planes. The traceback (linear-space in the cube's length) runs in two phases:
 * a forward pass keeps one plane per slab boundary and no codes; then each slab from the top
 * down recomputes its codes from the plane below it, and the walk continues through it.
 * Scores and alignments are identical to the one-launch path. Errors: EINVAL (null). */
trioseq_status trioseq_batch_slabs(trioseq_batch_t batch, int32_t* slices, int32_t* slabs);

/* Release a device-resident batch. Null is accepted. The call waits for the batch's own last
 * trioseq_batch_run (an event recorded on the stream that run was given) and synchronises no
 * other stream; the batch's memory is freed in the order of its private stream. */
trioseq_status trioseq_batch_destroy(trioseq_batch_t batch);

/* trioseq_batch_profile — when enable != 0, each trioseq_batch_run records CUDA events on its
 * stream around the wavefront kernel and around the traceback walk. trioseq_batch_timing then
 * returns, after trioseq_batch_scores (or a stream synchronisation), ms[0] = wavefront kernel
 * time and ms[1] = walk time (0 in score-only mode) of the last run.
 * Errors: EINVAL (null, profiling off or no run yet), ECUDA. */
trioseq_status trioseq_batch_profile(trioseq_batch_t batch, int32_t enable);
trioseq_status trioseq_batch_timing(trioseq_batch_t batch, float ms[2]);

/* trioseq_plan_autotune — pick the kernel variant for a class of work by measuring it.
 * Runs the sample batch (host strings, n >= 1, mode as for trioseq_align_batch) once per
 * candidate — every instantiated register tile per lane (8x8, 4x8, 4x4 cells, i.e. column blocks
 * of 32x64, 16x64 and 16x32 cells per warp, and in traceback mode also 8x4, 32x32 cells; in
 * score-only global mode with every sigma'' in [0, 33] also the two-cells-per-register tiles
 * 8x16 and 8x8v, 32x128 and 32x64 cells per warp) times
 * progress intervals of 4, 8, 16 and 32 steps —
 * times two passes of each with CUDA events on the legacy default stream, and remembers the
 * fastest in the plan for batches of the same mode, the same single-or-batch kind, and the same
 * bit length of the longest sequence. Later batches of that class use it; other classes keep
 * the defaults (8x8 score-only, 4x8 traceback, interval 8). Outputs (any may be null) report
 * the choice. The plan's device memory is untouched; a temporary workspace is used.
 * Errors: EINVAL, EOVERFLOW, ENOMEM, ETIMEOUT, ECUDA. */
trioseq_status trioseq_plan_autotune(trioseq_plan_t plan, const trioseq_triplet* sample, size_t n,
                                     uint32_t mode, int32_t* tile_j, int32_t* tile_k,
                                     int32_t* ti);

/* Bytes copied host->device (encoded inputs, descriptors, queue) and device->host (scores,
 * error word, alignments) by the last trioseq_align_batch call on this plan. */
trioseq_status trioseq_plan_io_bytes(trioseq_plan_t plan, uint64_t* h2d, uint64_t* d2h);

/* ---- serving: continuous batching behind submit/poll ---- */

typedef struct trioseq_server_s* trioseq_server_t;

/* trioseq_server_create — start a server thread that owns a pending queue and admits requests
 * by device memory and free slots, re-batching them each tick into launches on several CUDA
 * streams so that work of different requests overlaps on the device.
 * Admission: the workspace estimates of all launches on the device together stay within
 * `hbm_budget` bytes (0 = 80% of the memory free at creation, and then each admission is also
 * bounded by the memory free on the device at that moment). One launch groups same-scheme,
 * same-mode requests up to a quarter of the budget; a single larger request (up to the whole
 * budget; a global-type triplet counted at its slab workspace, see trioseq_batch_slabs) waits in
 * arrival order until the running launches leave it room. A request larger than the budget
 * completes with ENOMEM (reported by trioseq_poll).
 * plans[0..nplans) are the scoring schemes a request may name by index (e.g. 0 = DNA,
 * 1 = protein); they must outlive the server.
 * Errors: EINVAL, ENOMEM, ECUDA. */
trioseq_status trioseq_server_create(const trioseq_plan_t* plans, int32_t nplans,
                                     size_t hbm_budget, trioseq_server_t* out);

/* trioseq_submit — enqueue one triplet (copied before return) under plan index `plan_id` with
 * `mode`; returns a ticket. Non-blocking. Errors: EINVAL, EAGAIN (queue full), EOVERFLOW. */
trioseq_status trioseq_submit(trioseq_server_t srv, const trioseq_triplet* triplet,
                              int32_t plan_id, uint32_t mode, uint64_t* ticket);

/* trioseq_poll — non-blocking. EAGAIN while the request is pending; OK once done, with *score
 * set and, for traceback requests, rows[0..2] filled (cap bytes each, *aln_len set; rows may be
 * null for score-only requests). A ticket is consumed by the first OK. Errors: EINVAL (unknown
 * ticket, cap too small), ETIMEOUT / ECUDA (the request's launch failed). */
trioseq_status trioseq_poll(trioseq_server_t srv, uint64_t ticket, int32_t* score, char* rows[3],
                            size_t cap, size_t* aln_len);

/* Stop the server thread after finishing admitted work and release it. */
trioseq_status trioseq_server_destroy(trioseq_server_t srv);

/* ---- multi-GPU work partitioning (host only) ---- */

enum { TRIOSEQ_PART_BLOCKED = 0, TRIOSEQ_PART_INTERLEAVED = 1, TRIOSEQ_PART_DYNAMIC = 2,
       TRIOSEQ_PART_LARGEST_FIRST = 3 };

/* trioseq_partition — assign each triplet of a set to one of nranks ranks (one rank per GPU, each
 * aligning its share with its own plan), by the three schemes of Sec. V-D:
 *   TRIOSEQ_PART_BLOCKED     : contiguous chunks in dataset order; rank r gets triplets
 *                              floor(r*n/nranks) .. floor((r+1)*n/nranks) - 1 (the paper gives
 *                              no chunk rule; sizes differ by at most one);
 *   TRIOSEQ_PART_INTERLEAVED : round robin, triplet t to rank t mod nranks;
 *   TRIOSEQ_PART_DYNAMIC     : in dataset order, each triplet to the rank with the least
 *                              cumulative cell count so far (ties: lowest rank).
 *   TRIOSEQ_PART_LARGEST_FIRST : the dynamic rule applied to the triplets in order of
 *                              decreasing cell count, ties in dataset order (LPT list
 *                              scheduling; not in the paper). Its largest load is at most
 *                              4/3 - 1/(3 nranks) times the optimum.
 * A triplet's work is the paper's cell count |S0|*|S1|*|S2|.
 *   lens           : host array of 3n lengths, triplet t at lens[3t .. 3t+2] (caller-owned).
 *   rank_of        : out, host array of n ranks in [0, nranks) (caller-owned).
 *   cells_per_rank : out, host array of nranks cumulative cell counts; may be null.
 * Pure host computation: needs no GPU and no plan, allocates O(nranks) host memory, writes no
 * output on error. There is no collective: every rank computes the same partition from the
 * same lengths and keeps its own triplets.
 * Errors: EINVAL (nranks < 1 or > 2^20, unknown scheme, null lens or rank_of with n > 0),
 * ENOMEM (host allocation), EOVERFLOW (the
 * set's total cell count exceeds 2^64 - 1). */
trioseq_status trioseq_partition(const uint32_t* lens, size_t n, int32_t nranks, int32_t scheme,
                                 int32_t* rank_of, uint64_t* cells_per_rank);

/* ---- measurement ---- */

/* trioseq_alu_rate — measured rate of one int32 instruction form on the current GPU. It backs the
 * roofline of the cell recurrence (Eq. 1, Sec. II): the engine counts 13 int32 operations per
 * cell (7 adds, 6 maxima) against SMs x 128 int32 lanes x SM clock, and issues them as the forms
 * below. The paper has no counterpart; this call measures the hardware.
 *   op             : 0 max(x, y); 1 max(y + b, x) (__viaddmax_s32, two operations);
 *                    2 max(x, y, z) (__vimax3_s32, two operations); 3 x + y + b (two operations);
 *                    4 y * one + x with a runtime one (the FMA-pipe add).
 *   per_clk_per_sm : out, thread-level instructions of that form completed per SM clock per SM,
 *                    with every SM fully occupied by independent recurrences.
 *   sm_mhz         : out, the SM clock during the measurement (cycles / event time).
 * Allocates a few MB of device memory for the duration of the call and launches two short
 * kernels (~0.1 s). Errors: TRIOSEQ_EINVAL (op out of range, null output), TRIOSEQ_ECUDA. */
trioseq_status trioseq_alu_rate(int32_t op, double* per_clk_per_sm, double* sm_mhz);

/* ---- allocation-free entry point ---- */

/* trioseq_align_noalloc — score one triplet without allocating any memory in the call.
 * (The paper has no counterpart: this is an integration entry point of this library.)
 * For callers that cannot call cudaMalloc when they align: processes whose device memory is
 * already fully reserved by another allocator (a framework's caching pool, a serving process
 * with a fixed memory budget) or plugin hosts that forbid allocation inside their callbacks.
 * The call places its whole workspace (encoded residues, descriptor, work queue, progress
 * flags, boundary records) in one 64 MiB array in device memory that the library declares at
 * file scope; every GPU that loads the library holds that array until the process exits.
 *   scoring   : host scoring scheme as for trioseq_plan (validated in the call).
 *   d_s0/1/2  : caller-owned DEVICE buffers of a, b, c bytes (alphabet characters, not codes);
 *               may be null when the length is 0.
 *   d_score   : caller-owned DEVICE int32 that receives the optimal global score.
 *   stream    : cudaStream_t (NULL = legacy default); the call synchronises it before
 *               returning, so the score is ready on return.
 * Same score as trioseq_align_batch in TRIOSEQ_SCORE_ONLY mode (score only, no traceback).
 * The first call on a device looks up the array's device address (make it before any stream
 * capture). All calls share the array and it keeps the last call's contents; each call clears
 * what must start at zero, and calls that overlap on the GPU (other streams, other threads)
 * race, so callers serialise them.
 * Errors: ESCRATCH (the triplet's workspace exceeds the 64 MiB array: roughly a*b*c > 3e8 for
 * DNA-sized tiles), EINVAL (null pointers, bad scoring, a byte outside the alphabet),
 * EOVERFLOW, ETIMEOUT, ECUDA. */
trioseq_status trioseq_align_noalloc(const trioseq_scoring* scoring, const unsigned char* d_s0,
                                     uint32_t a, const unsigned char* d_s1, uint32_t b,
                                     const unsigned char* d_s2, uint32_t c, int32_t* d_score,
                                     void* stream);

/* Human-readable name of a status code (static storage). */
const char* trioseq_strerror(trioseq_status st);

#ifdef __cplusplus
}
#endif

#endif /* TRIOSEQ_H */

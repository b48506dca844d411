// runtime.cu — host runtime behind the C ABI of include/trioseq.h.
//
// Plan: scoring scheme validated and turned into the device tables of the shifted frame
// (sigma'' = sigma - 2*alpha, a virtual residue row/column of zeros, x8 for traceback keys).
// Batch: encoded + packed residues, per-triplet descriptors (engine.h), the ordered column-task
// queue, and a device workspace (faces, progress flags, codes, outputs).
// Queue order: tasks sorted by anti-diagonal D = J + K of their column block, then by the
// triplet's rank in longest-processing-time order (largest cube first). Every producer of a
// task, (J-1,K) and (J,K-1), has a smaller D and therefore an earlier queue slot. The LPT part
// follows the paper's dynamic partition by cumulative cells (Sec. V-D), applied here to the
// warps of one GPU instead of to GPUs.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "engine.h"
#include "guard.h"
#include "trioseq.h"

using namespace trioseq;

namespace {

// NVTX range for the duration of a scope: plan, autotune, batch, run, traceback and server
// launches show up by name in profilers that read NVTX (header-only NVTX 3; no cost without one).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Host-side fault injection for tests: with TRIOSEQ_TEST_FAIL_ALLOC=N at trioseq_plan, the N-th
// device allocation after it fails as if the device were out of memory.
std::atomic<long> g_alloc_calls{0};
std::atomic<long> g_alloc_fail_at{0};

bool injected_alloc_failure() {
  const long at = g_alloc_fail_at.load(std::memory_order_relaxed);
  return at > 0 && g_alloc_calls.fetch_add(1, std::memory_order_relaxed) + 1 == at;
}

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaStream_t st_ = nullptr;  // stream of a stream-ordered allocation (freed in its order)
  ~DevBuf() { reset(); }
  // Release the buffer: stream-ordered allocations are freed in their stream's order, which
  // blocks neither the host nor other streams.
  void reset() {
    if (p) {
      if (st_)
        cudaFreeAsync(p, st_);
      else
        cudaFree(p);
    }
    p = nullptr;
    cap = 0;
    st_ = nullptr;
  }
  // Grow to at least `bytes` (contents are not preserved). With a stream, the old buffer is
  // released and the new one taken in that stream's order (no device-wide synchronisation), so
  // a growing workspace does not stall work running on other streams. The caller orders that
  // stream after the old buffer's last use.
  bool ensure(size_t bytes, cudaStream_t st = nullptr) {
    if (bytes <= cap && p) return true;
    const size_t want = std::max<size_t>(bytes, 256);
    if (injected_alloc_failure()) return false;
    reset();
    const cudaError_t e = st ? cudaMallocAsync(&p, want, st) : cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return false;
    }
    cap = want;
    st_ = st;
    return true;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

struct HostPinned {
  void* p = nullptr;
  size_t cap = 0;
  ~HostPinned() {
    if (p) cudaFreeHost(p);
  }
  bool ensure(size_t bytes) {
    if (bytes <= cap && p) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max<size_t>(bytes, 4096);
    if (cudaMallocHost(&p, want) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cap = want;
    return true;
  }
};

// Device workspace of one in-flight batch.
struct Workspace {
  DevBuf inputs;    // packed residues | descriptors | tasks | traceback tables
  DevBuf faces;     // j- and k-face planes
  DevBuf progress;  // progress flags | queue head | error word
  DevBuf codes;     // traceback codes
  DevBuf scores;    // int32 per triplet
  DevBuf rows;      // traceback rows
  DevBuf lens;      // alignment lengths
  DevBuf planes;    // slab mode: checkpoint planes (traceback) or two ping-pong planes (score)
  DevBuf walkstate; // slab mode: (i, j, k, n) of the traceback walk between slabs
  DevBuf best64;    // semi-global / local traceback: (score, first cell) key per triplet
  DevBuf spans;     // traceback: begin and end cell of each alignment (6 int32)
  HostPinned staging;
  // Buffers are allocated and freed in this stream's order. Plans and device-resident batches
  // own a private stream here (own_stream); a serving slot uses its launch stream.
  cudaStream_t alloc_stream = nullptr;
  bool own_stream = false;
  // Recorded on the launching stream after each enqueued use: growth and destruction wait for
  // this workspace's own work only, never for the whole device.
  cudaEvent_t last_use = nullptr;
  bool used = false;

  // A private allocation stream (non-blocking, so it never waits on the legacy default stream).
  cudaError_t make_own_stream() {
    const cudaError_t e = cudaStreamCreateWithFlags(&alloc_stream, cudaStreamNonBlocking);
    own_stream = e == cudaSuccess;
    if (e != cudaSuccess) alloc_stream = nullptr;
    return e;
  }
  // Mark the end of a use enqueued on `st`.
  cudaError_t mark_use(cudaStream_t st) {
    if (!last_use) {
      const cudaError_t e = cudaEventCreateWithFlags(&last_use, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        last_use = nullptr;
        return e;
      }
    }
    const cudaError_t e = cudaEventRecord(last_use, st);
    used = used || e == cudaSuccess;
    return e;
  }
  // Host wait for this workspace's last recorded use (not for other streams' work).
  void wait_last_use() {
    if (used && last_use) cudaEventSynchronize(last_use);
  }
  // Order the allocation stream after the last recorded use, before buffers are freed there.
  void order_after_last_use() {
    if (used && last_use && alloc_stream) cudaStreamWaitEvent(alloc_stream, last_use, 0);
  }
  // Free every device buffer in the allocation stream's order, after the last recorded use.
  // Must run while that stream exists (a serving slot calls it before destroying its stream).
  void release() {
    order_after_last_use();
    for (DevBuf* b : {&inputs, &faces, &progress, &codes, &scores, &rows, &lens, &planes,
                      &walkstate, &best64, &spans})
      b->reset();
  }
  ~Workspace() {
    release();
    if (last_use) cudaEventDestroy(last_use);
    if (own_stream && alloc_stream) cudaStreamDestroy(alloc_stream);  // released when idle
  }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Register tile per lane: nj x nk cells; vl = 1 for the two-cells-per-register kernel
// (wavefront_vl.cuh), whose lane tile is two nj x nk/2 column halves.
struct Variant {
  int nj, nk;
  int vl = 0;
};

}  // namespace

struct trioseq_plan_s {
  int device = 0;
  int sms = 0;
  int K = 0;
  int KP = 0;
  char alphabet[kMaxAlphabet] = {};
  int16_t lut[256];
  std::vector<int32_t> sub;
  int32_t gap = 0;
  int atype = kGlobal;             // alignment type of Sec. II (plan flags)
  int32_t max_abs_sig2 = 0;        // max |sigma''| over the extended table
  DevBuf sig_score, sig_tb;        // KP*KP int32 device tables
  bool affine = false;             // trioseq_plan_affine: natural affine gap costs (affine.cu)
  int32_t gap_open = 0;            // gamma, per maximal gap run of a pair
  DevBuf sig_affine;               // KP*KP int32 table of sigma itself (affine model)
  int32_t max_abs_sub = 0;         // max |sigma|
  Workspace ws;                    // workspace of trioseq_align_batch
  std::unique_ptr<trioseq_batch_s> last;  // last align_batch (traceback rows kept here)
  int TI = 8;
  int64_t wait_ns = 2000000000LL;  // 2 s without progress = give up
  bool test_wait_unset = false;    // test switch: first-wave warps wait on a flag nothing sets
  bool test_poison = false;        // test switch: boundary records start as a large garbage value
  int data_flags = -1;             // TRIOSEQ_DATA_FLAGS: records as readiness flags (-1: chosen)
  bool graphs = true;              // trioseq_batch_run replays a captured CUDA graph
  bool packed16 = true;            // pair score-only global triplets in int16 halves if they fit
  bool sig2_nonneg = false;        // every sigma'' >= 0: the biased packed mode applies
  size_t slab_budget = 0;          // bytes a one-triplet batch may use before it runs in slabs
  bool pace = true;                // pace the first wave of multi-wave launches
  int slab_slices = 0;             // forced slab height (0: chosen from the budget)
  Variant score_variant{8, 8};
  Variant tb_variant{4, 8};
  // Autotuner cache: (mode, single triplet or batch, bit length of the longest sequence) ->
  // fastest (tile, progress interval) measured by trioseq_plan_autotune.
  struct Tuned {
    Variant var;
    int TI;
  };
  std::map<int, Tuned> tuned;
  bool tuning = false;     // set while the autotuner forces candidates
  Tuned forced{{8, 8}, 8};
};

namespace {
int tune_key(uint32_t mode, size_t n, uint32_t maxlen) {
  int bits = 0;
  while ((maxlen >> bits) > 0 && bits < 31) ++bits;
  return (int)mode * 1000 + (n > 1 ? 100 : 0) + bits;
}
}  // namespace

struct trioseq_batch_s {
  trioseq_plan_s* plan = nullptr;
  Workspace* ws = nullptr;             // where it runs (owned if own_ws)
  std::unique_ptr<Workspace> own_ws;
  size_t n = 0;
  uint32_t mode = 0;
  Variant var{8, 8};
  uint64_t cells = 0;
  std::vector<TripDesc> desc;
  std::vector<Task> tasks;
  std::vector<int32_t> tb_trips;       // triplet index per traceback request
  std::vector<int64_t> row_off;
  std::vector<int32_t> row_cap;
  std::vector<int32_t> tb_of;          // triplet -> traceback request (-1)
  std::vector<int8_t> seq;             // packed residue codes (host copy)
  size_t seq_bytes = 0, face_ints = 0, code_words = 0, rows_bytes = 0;
  size_t off_desc = 0, off_tasks = 0, off_tb = 0, off_rowoff = 0, off_rowcap = 0, inputs_bytes = 0;
  int grid = 0;
  size_t smem = 0;
  int TI = 8;  // progress-publication interval of this batch's launches
  int packed = 0;  // packed int16x2 mode (0: none, 1: signed, 2: biased): two triplets per task
  int64_t affine_cells = 0;  // affine model: cells of the largest (j, k) plane
  // Slab mode (one triplet whose records, or codes, would not fit at once): the cube runs as
  // nslab launches of `slab` slices, chained through planes of plane_ints int32 each.
  int slab = 0, nslab = 0;
  size_t plane_ints = 0, nplanes = 0, off_slab = 0;
  std::vector<TripDesc> slab_desc;
  bool uploaded = false;
  // results of the last run (host)
  std::vector<uint8_t> h_rows;
  std::vector<int32_t> h_lens;
  std::vector<int32_t> h_spans;  // 6 per traceback request
  bool have_rows = false;
  // optional per-kernel timing (events on the launching stream)
  bool profile = false;
  bool timed = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  uint64_t h2d_bytes = 0, d2h_bytes = 0;
  // trioseq_batch_run replays one captured CUDA graph (progress reset, wavefront, walk). The key
  // holds the buffer addresses and the profiling switch the graph was captured with.
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::array<const void*, 12> gkey{};
  ~trioseq_batch_s() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

trioseq_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TRIOSEQ_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TRIOSEQ_ENOMEM : TRIOSEQ_ECUDA;
}

int env_int(const char* name, int def) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : def;
}

// Device layout of a batch's input block: residues | descriptors | slab descriptors | queue |
// traceback tables.
void layout_inputs(trioseq_batch_s* bt) {
  size_t off = align_up(bt->seq_bytes, 256);
  bt->off_desc = off;
  off = align_up(off + sizeof(TripDesc) * std::max<size_t>(bt->n, 1), 256);
  bt->off_slab = off;
  off = align_up(off + sizeof(TripDesc) * bt->slab_desc.size(), 256);
  bt->off_tasks = off;
  off = align_up(off + sizeof(Task) * std::max<size_t>(bt->tasks.size(), 1), 256);
  bt->off_tb = off;
  off = align_up(off + sizeof(int32_t) * std::max<size_t>(bt->tb_trips.size(), 1), 256);
  bt->off_rowoff = off;
  off = align_up(off + sizeof(int64_t) * std::max<size_t>(bt->row_off.size(), 1), 256);
  bt->off_rowcap = off;
  off = align_up(off + sizeof(int32_t) * std::max<size_t>(bt->row_cap.size(), 1), 256);
  bt->inputs_bytes = off;
}

// Affine-gap batch (affine.cu): one queue entry per triplet, largest cube first; each CTA of
// the persistent launch sweeps its triplets' anti-diagonal planes in four rotating plane
// buffers of 13 int32 states per cell. Score only.
trioseq_status build_affine(trioseq_plan_s* plan, trioseq_batch_s* bt) {
  const size_t n = bt->n;
  std::vector<int32_t> order(n);
  int64_t maxcells = 1;
  for (size_t t = 0; t < n; t++) {
    order[t] = (int32_t)t;
    const TripDesc& d = bt->desc[t];
    maxcells = std::max<int64_t>(maxcells, (int64_t)(d.len[1] + 1) * (d.len[2] + 1));
  }
  const auto vol = [&](int32_t t) {
    const TripDesc& d = bt->desc[t];
    return (double)(d.len[0] + 1) * (d.len[1] + 1) * (d.len[2] + 1);
  };
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return vol(x) > vol(y); });
  bt->tasks.clear();
  for (const int32_t t : order) bt->tasks.push_back(Task{t, 0, 0, 0});
  int bpm = 0;
  if (affine_occupancy(&bpm) != 0 || bpm <= 0) return TRIOSEQ_ECUDA;
  bt->grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)plan->sms * bpm, n));
  bt->affine_cells = maxcells;
  bt->face_ints = (size_t)bt->grid * 4 * (size_t)maxcells * 16;  // 16 int32 per cell (13 used)
  bt->seq_bytes = bt->seq.size();
  layout_inputs(bt);
  return TRIOSEQ_OK;
}

// Build the host side of a batch: encode, pack, describe, order the queue.
trioseq_status build_batch(trioseq_plan_s* plan, const trioseq_triplet* trip, size_t n,
                           uint32_t mode, trioseq_batch_s* bt) {
  if (!trip && n) return TRIOSEQ_EINVAL;
  if (mode > TRIOSEQ_WITH_TRACEBACK) return TRIOSEQ_EINVAL;
  const bool tb = mode == TRIOSEQ_WITH_TRACEBACK;
  bt->plan = plan;
  bt->n = n;
  bt->mode = mode;
  bt->var = tb ? plan->tb_variant : plan->score_variant;
  bt->TI = plan->TI;
  {
    uint32_t maxlen = 0;
    for (size_t t = 0; t < n; t++)
      for (int q = 0; q < 3; q++) maxlen = std::max(maxlen, trip[t].len[q]);
    if (plan->tuning) {
      bt->var = plan->forced.var;
      bt->TI = plan->forced.TI;
    } else {
      auto it = plan->tuned.find(tune_key(mode, n, maxlen));
      if (it != plan->tuned.end()) {
        bt->var = it->second.var;
        bt->TI = it->second.TI;
      }
    }
  }
  // Two cells of one triplet per register (wavefront_vl.cuh), variants 8x16 and 8x8v: score-only
  // alignment of any type with every sigma'' >= 0, max sigma'' <= 33 (the kernel's range
  // argument),
  // and boundary records within the slab budget (it has no slab form). Outside the autotuner's
  // own candidate runs, work it cannot take runs on the int32 8x8 kernel instead.
  if (bt->var.vl) {
    // (semi-global and local too: their zero axes and floor add steps of -2*alpha, which must
    // also stay <= 33)
    bool ok_vl = !tb && plan->sig2_nonneg && plan->max_abs_sig2 <= 33 &&
                 (plan->atype == kGlobal || -2 * plan->gap <= 33) &&
                 wavefront_vl(bt->var.nj, bt->var.nk, bt->var.vl - 1, plan->atype) != nullptr;
    if (ok_vl) {
      const int wj = kPR * bt->var.nj, wk = kPC * bt->var.nk;
      double rec = 0;  // int32 boundary records of all triplets: (a+1) x tasks x (WK+4 + WJ)
      for (size_t t = 0; t < n; t++)
        rec += (trip[t].len[0] + 1.0) * ((trip[t].len[1] + wj) / wj) *
               ((trip[t].len[2] + wk) / wk) * (4.0 * (wk + 4 + wj));
      ok_vl = rec <= (double)plan->slab_budget;
    }
    if (!ok_vl) {
      if (plan->tuning) return TRIOSEQ_ECUDA;  // the autotuner skips the candidate
      bt->var = Variant{8, 8};
    }
  }
  const int NJ = bt->var.nj, NK = bt->var.nk;
  const int WJ = kPR * NJ, WK = kPC * NK, W = NJ * NK / 8;
  // encode + pack (16-byte aligned sequences)
  size_t total = 0;
  for (size_t t = 0; t < n; t++)
    for (int q = 0; q < 3; q++) {
      if (trip[t].len[q] && !trip[t].s[q]) return TRIOSEQ_EINVAL;
      if (trip[t].len[q] > (1u << 24)) return TRIOSEQ_EOVERFLOW;
      total += align_up(trip[t].len[q], 16);
    }
  bt->seq.assign(std::max<size_t>(total, 16), 0);
  bt->desc.resize(n);
  bt->tb_of.assign(n, -1);
  bt->tb_trips.clear();
  bt->row_off.clear();
  bt->row_cap.clear();
  size_t pos = 0, face = 0, codes = 0, rows = 0;
  int64_t prog = 0;
  bt->cells = 0;
  // 1a. Packed positions, then the residue codes (alphabet lookup). Large batches encode on
  //     several host threads, each over a contiguous range of triplets.
  for (size_t t = 0; t < n; t++)
    for (int q = 0; q < 3; q++) {
      bt->desc[t].s_off[q] = (int64_t)pos;
      pos += align_up(trip[t].len[q], 16);
    }
  {
    std::atomic<bool> bad{false};
    const auto encode = [&](size_t t0, size_t t1) {
      for (size_t t = t0; t < t1 && !bad.load(std::memory_order_relaxed); t++)
        for (int q = 0; q < 3; q++) {
          const unsigned char* src = reinterpret_cast<const unsigned char*>(trip[t].s[q]);
          int8_t* dst = bt->seq.data() + bt->desc[t].s_off[q];
          int16_t acc = 0;
          for (uint32_t e = 0; e < trip[t].len[q]; e++) {
            const int16_t code = plan->lut[src[e]];
            acc |= code;  // negative iff some residue is outside the alphabet
            dst[e] = (int8_t)code;
          }
          if (acc < 0) bad.store(true, std::memory_order_relaxed);
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nth = std::min<size_t>({(size_t)8, (size_t)hw, n, total / (1u << 19) + 1});
    if (nth <= 1) {
      encode(0, n);
    } else {  // split the triplets into nth ranges of about equal residue counts
      std::vector<std::thread> pool;
      size_t t0 = 0;
      for (size_t k = 1; k <= nth && t0 < n; k++) {
        size_t t1 = t0;
        const size_t goal = total * k / nth;
        while (t1 < n && (k == nth || (size_t)bt->desc[t1].s_off[0] < goal)) t1++;
        if (t1 == t0) continue;
        try {
          pool.emplace_back(encode, t0, t1);
        } catch (...) {  // no thread: encode the range here
          encode(t0, t1);
        }
        t0 = t1;
      }
      for (auto& th : pool) th.join();
    }
    if (bad.load()) return TRIOSEQ_EINVAL;
  }
  // 1b. Per triplet: range checks, output slots.
  for (size_t t = 0; t < n; t++) {
    TripDesc& d = bt->desc[t];
    int64_t sumlen = 0;
    for (int q = 0; q < 3; q++) {
      const uint32_t L = trip[t].len[q];
      d.len[q] = d.glen[q] = (int32_t)L;
      sumlen += L;
    }
    // |M'| <= max|sigma''| * (a+b+c) (and, with zero axes or v = 0, <= 2|alpha| * (a+b+c));
    // keys need 8*|M'| + 8 below 2^29.
    if ((int64_t)std::max(plan->max_abs_sig2, plan->atype != kGlobal ? -2 * plan->gap : 0) *
            sumlen >= (1LL << 26) - 1)
      return TRIOSEQ_EOVERFLOW;
    if (2LL * (int64_t)std::abs(plan->gap) * sumlen >= (1LL << 30)) return TRIOSEQ_EOVERFLOW;
    // semi-global / local traceback: the best cell's index must fit 37 bits (engine.h, best64)
    if (tb && plan->atype != kGlobal &&
        (double)(d.len[0] + 1) * (d.len[1] + 1) * (d.len[2] + 1) >= (double)(1ULL << 37))
      return TRIOSEQ_EOVERFLOW;
    // affine: |score| <= (3 max|sigma| + 3|alpha| + 3|gamma|) * (a+b+c), kept below 2^29
    if (plan->affine &&
        (int64_t)(3 * plan->max_abs_sub + 3 * std::abs(plan->gap) + 3 * std::abs(plan->gap_open)) *
                std::max<int64_t>(sumlen, 1) >= (1LL << 29))
      return TRIOSEQ_EOVERFLOW;
    d.pair = -1;
    d.score_base = 2 * plan->gap * (int32_t)sumlen;
    d.out_idx = (int32_t)t;
    d.tb_idx = -1;
    d.code_off = -1;
    bt->cells += (uint64_t)d.len[0] * (uint64_t)d.len[1] * (uint64_t)d.len[2];
  }
  if (plan->affine) {
    if (tb) return TRIOSEQ_ENOTIMPL;  // the affine model is score-only on the device
    return build_affine(plan, bt);
  }
  // 2. Units of work: one triplet, or in packed int16x2 mode two triplets of the same column-task
  //    grid class paired in one unit (the high halves run on the grid of their maximal lengths).
  //    Packing needs every value of the pair's grid within the int16 margin of engine.h:
  //    max|sigma''| * (a+b+c + 3) < 2^14 on the grid's lengths.
  std::vector<std::pair<int32_t, int32_t>> units;  // (low-half triplet, high-half triplet or -1)
  bt->packed = 0;
  const bool vl = bt->var.vl != 0;  // admitted above
  if (vl) bt->packed = 2 + bt->var.vl;  // 3: registers; 4, 5: sigma'' tile in shared memory
  const int pmode = plan->sig2_nonneg ? 2 : 1;
  if (!vl && !tb && plan->atype == kGlobal && plan->packed16 && n >= 2 &&
      wavefront_packed(NJ, NK, pmode) != nullptr) {
    std::vector<int32_t> order(n);
    for (size_t t = 0; t < n; t++) order[t] = (int32_t)t;
    const auto cls = [&](int32_t t) {
      const TripDesc& d = bt->desc[t];
      return std::make_tuple((d.len[1] + WJ) / WJ, (d.len[2] + WK) / WK, d.len[0]);
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return cls(x) < cls(y); });
    bool fits = true;
    for (size_t u = 0; u < n && fits; u += 2) {
      const int32_t t0 = order[u], t1 = (u + 1 < n) ? order[u + 1] : order[u];
      int64_t gsum = 0;
      for (int q = 0; q < 3; q++)
        gsum += std::max(bt->desc[t0].len[q], bt->desc[t1].len[q]);
      fits = (int64_t)plan->max_abs_sig2 * (gsum + 3) < (1 << 14);
      units.emplace_back(t0, t1);
    }
    if (fits) {
      bt->packed = pmode;
    } else {
      units.clear();
    }
  }
  if (units.empty())  // one unit per triplet (no pairs formed)
    for (size_t t = 0; t < n; t++) units.emplace_back((int32_t)t, -1);
  // 3. Per unit: task grid, boundary records, progress flags, traceback codes and rows.
  for (const auto& un : units) {
    TripDesc& d = bt->desc[un.first];
    if (un.second >= 0) {
      const TripDesc& h = bt->desc[un.second];
      for (int q = 0; q < 3; q++) d.glen[q] = std::max(d.len[q], h.len[q]);
      d.pair = un.second;
    }
    const int a = d.glen[0], b = d.glen[1], c = d.glen[2];
    d.nJ = (b + 1 + WJ - 1) / WJ;
    d.nK = (c + 1 + WK - 1) / WK;
    d.T = a + 1 + (kPR - 1) + (kPC - 1) + (vl ? kPC : 0);  // vl: 2*kPC virtual lane columns
    // boundary records of every column task: (a+1) x (WK+4) j-records, (a+1) x WJ k-records
    const size_t ntask = (size_t)d.nJ * (size_t)d.nK;
    d.oj_off = (int64_t)face;
    face += ntask * (size_t)(a + 1) * (size_t)(WK + 4);
    d.ok_off = (int64_t)face;
    face += ntask * (size_t)(a + 1) * (size_t)WJ;
    face = align_up(face, 4);
    d.prog_base = prog;
    prog += (int64_t)d.nJ * d.nK;
    if (un.second >= 0 && un.second != un.first) {  // the high half shares the grid
      TripDesc& h = bt->desc[un.second];
      for (int q = 0; q < 3; q++) h.glen[q] = d.glen[q];
      h.nJ = d.nJ;
      h.nK = d.nK;
      h.T = d.T;
      h.oj_off = d.oj_off;
      h.ok_off = d.ok_off;
      h.prog_base = d.prog_base;
    }
    if (tb) {
      const int32_t t = un.first;
      d.code_off = (int64_t)codes;
      codes += (size_t)d.nJ * d.nK * (size_t)d.T * 32 * W;
      d.tb_idx = (int32_t)bt->tb_trips.size();
      bt->tb_of[t] = d.tb_idx;
      bt->tb_trips.push_back(t);
      const int cap = std::max(1, a + b + c);
      bt->row_off.push_back((int64_t)rows);
      bt->row_cap.push_back(cap);
      rows += align_up((size_t)3 * cap, 16);
    }
  }
  // 4. Slab mode: one global-type int32 triplet whose boundary records (and, with traceback,
  //    codes) would exceed the plan's budget at once, or any such triplet when a slab height is
  //    forced. The cube then runs slab by slab, each launch seeded from the plane the slab below
  //    left (DESIGN: linear-space traceback).
  bt->slab = bt->nslab = 0;
  bt->nplanes = bt->plane_ints = 0;
  bt->slab_desc.clear();
  if (n == 1 && plan->atype == kGlobal && !bt->packed) {
    TripDesc& d = bt->desc[0];
    const size_t ntask = (size_t)d.nJ * (size_t)d.nK;
    const size_t A = (size_t)d.len[0] + 1;                     // slices of the cube
    const size_t rec = ntask * (size_t)((WK + 4) + WJ);         // record ints per slice
    const size_t cw = tb ? ntask * 32 * (size_t)W : 0;          // code words per step
    const size_t plane = (size_t)d.nJ * WJ * (size_t)d.nK * WK;  // ints per plane
    const auto bytes = [&](size_t S) {  // workspace of slab height S
      const size_t slabs = (A + S - 1) / S;
      const size_t planes = tb ? slabs - 1 : std::min<size_t>(2, slabs - 1);
      return 4 * (S * rec + (S + 10) * cw + planes * plane);
    };
    size_t S = (size_t)plan->slab_slices;
    if (S == 0 && 4 * (A * rec + (A + 10) * cw) > plan->slab_budget) {
      // the largest power-of-two fraction of the cube that fits; fall back to the smallest
      // workspace when none does (the allocation then reports ENOMEM)
      size_t best = A;
      for (S = A; S >= 1; S = S / 2) {
        if (bytes(S) < bytes(best)) best = S;
        if (bytes(S) <= plan->slab_budget) break;
        if (S == 1) {
          S = best;
          break;
        }
      }
    }
    if (S > 0) {
      S = std::min(S, A);
      bt->slab = (int)S;
      bt->nslab = (int)((A + S - 1) / S);
      bt->plane_ints = plane;
      bt->nplanes = tb ? bt->nslab - 1 : std::min(2, bt->nslab - 1);
      for (int m = 0; m < bt->nslab; m++) {
        TripDesc sd = d;
        const int len0 = (int)std::min(S, A - (size_t)m * S) - 1;  // last local slice
        sd.len[0] = sd.glen[0] = len0;
        sd.T = len0 + 1 + (kPR - 1) + (kPC - 1);
        sd.oj_off = 0;
        sd.ok_off = (int64_t)(ntask * S * (size_t)(WK + 4));
        sd.prog_base = 0;
        sd.code_off = 0;
        sd.out_idx = (m == bt->nslab - 1) ? 0 : -1;  // only the top slab ends at (a, b, c)
        bt->slab_desc.push_back(sd);
      }
      d.code_off = 0;  // the walk reads the one slab of codes in the buffer
      face = ntask * S * (size_t)((WK + 4) + WJ);
      codes = tb ? ntask * (S + 10) * 32 * (size_t)W : 0;
    }
  }
  bt->seq_bytes = bt->seq.size();
  bt->face_ints = std::max<size_t>(face, 4);
  bt->code_words = std::max<size_t>(codes, 4);
  bt->rows_bytes = std::max<size_t>(rows, 16);
  // queue: (anti-diagonal, LPT rank of the unit's grid, J), built by counting sort on the
  // anti-diagonal: units visited in LPT order and J ascending within a unit give the same order as
  // a stable sort on the full key.
  const size_t nu = units.size();
  std::vector<int32_t> order(nu);
  for (size_t u = 0; u < nu; u++) order[u] = (int32_t)u;
  {
    const auto vol = [&](int32_t u) {
      const TripDesc& d = bt->desc[units[u].first];
      return (double)(d.glen[0] + 1) * (d.glen[1] + 1) * (d.glen[2] + 1);
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return vol(x) > vol(y); });
  }
  int maxD = 0;
  for (const auto& un : units) {
    const TripDesc& d = bt->desc[un.first];
    maxD = std::max(maxD, d.nJ + d.nK - 2);
  }
  std::vector<size_t> start((size_t)maxD + 2, 0);
  for (const auto& un : units) {
    const TripDesc& d = bt->desc[un.first];
    for (int J = 0; J < d.nJ; J++)
      for (int K = 0; K < d.nK; K++) start[(size_t)(J + K) + 1]++;
  }
  for (size_t D = 1; D < start.size(); D++) start[D] += start[D - 1];
  bt->tasks.assign((size_t)prog, Task{0, 0, 0, 0});
  {
    for (const int32_t u : order) {
      const int32_t t = units[u].first;
      const TripDesc& d = bt->desc[t];
      for (int J = 0; J < d.nJ; J++)
        for (int K = 0; K < d.nK; K++) bt->tasks[start[(size_t)(J + K)]++] = Task{t, J, K, 0};
    }
  }
  layout_inputs(bt);
  // launch shape
  bt->smem = bt->packed >= 3 ? wavefront_vl_smem_bytes(NJ, NK, plan->KP, bt->packed - 3)
                             : wavefront_smem_bytes(NJ, NK, plan->KP, bt->packed != 0);
  int bpm = 0;
  if (wavefront_occupancy(NJ, NK, tb, plan->atype, bt->packed, bt->slab > 0, bt->smem, &bpm) !=
          0 ||
      bpm <= 0)
    return TRIOSEQ_ECUDA;
  const int want = env_int("TRIOSEQ_CTAS_PER_SM", bpm);
  bt->grid = plan->sms * std::max(1, std::min(bpm, want));
  return TRIOSEQ_OK;
}

int plan_atype(const trioseq_batch_s* bt) { return bt->plan->atype; }

// Size the workspace and copy the inputs of `bt` into it (stream-ordered).
// `pinned`: stage through the workspace's pinned buffer and copy asynchronously on `st` (the
// per-call path); otherwise copy synchronously from pageable memory (one-off batch creation).
trioseq_status upload(trioseq_batch_s* bt, cudaStream_t st, bool pinned) {
  Workspace& ws = *bt->ws;
  const bool tb = bt->mode == TRIOSEQ_WITH_TRACEBACK;
  const size_t nprog = bt->tasks.size() + 64;
  cudaStream_t as = ws.alloc_stream;
  ws.order_after_last_use();  // a buffer that grows is freed only after its last use
  if (!ws.inputs.ensure(bt->inputs_bytes, as) ||
      !ws.faces.ensure(bt->face_ints * sizeof(int32_t), as) ||
      !ws.progress.ensure(nprog * sizeof(int32_t), as) ||
      !ws.scores.ensure(std::max<size_t>(bt->n, 1) * sizeof(int32_t), as) ||
      (tb && (!ws.codes.ensure(bt->code_words * sizeof(uint32_t), as) ||
              !ws.rows.ensure(bt->rows_bytes, as) ||
              !ws.lens.ensure(std::max<size_t>(bt->tb_trips.size(), 1) * sizeof(int32_t), as))) ||
      (bt->nplanes && !ws.planes.ensure(bt->nplanes * bt->plane_ints * sizeof(int32_t), as)) ||
      (bt->slab && tb && !ws.walkstate.ensure(4 * sizeof(int32_t), as)) ||
      (tb && !ws.spans.ensure(std::max<size_t>(bt->tb_trips.size(), 1) * 6 * sizeof(int32_t),
                              as)) ||
      (tb && plan_atype(bt) != kGlobal &&
       !ws.best64.ensure(std::max<size_t>(bt->n, 1) * sizeof(unsigned long long), as)) ||
      (pinned && !ws.staging.ensure(bt->inputs_bytes)))
    return TRIOSEQ_ENOMEM;
  // On a private allocation stream, the buffers are ready before any launch stream uses them.
  if (ws.own_stream && cudaStreamSynchronize(as) != cudaSuccess)
    return cuda_status(cudaGetLastError());
  std::vector<char> pageable;
  if (!pinned) pageable.assign(bt->inputs_bytes, 0);
  char* h = pinned ? reinterpret_cast<char*>(ws.staging.p) : pageable.data();
  std::memcpy(h, bt->seq.data(), bt->seq_bytes);
  std::memcpy(h + bt->off_desc, bt->desc.data(), sizeof(TripDesc) * bt->n);
  std::memcpy(h + bt->off_tasks, bt->tasks.data(), sizeof(Task) * bt->tasks.size());
  if (!bt->slab_desc.empty())
    std::memcpy(h + bt->off_slab, bt->slab_desc.data(), sizeof(TripDesc) * bt->slab_desc.size());
  if (tb) {
    std::memcpy(h + bt->off_tb, bt->tb_trips.data(), sizeof(int32_t) * bt->tb_trips.size());
    std::memcpy(h + bt->off_rowoff, bt->row_off.data(), sizeof(int64_t) * bt->row_off.size());
    std::memcpy(h + bt->off_rowcap, bt->row_cap.data(), sizeof(int32_t) * bt->row_cap.size());
  }
  cudaError_t e =
      pinned ? cudaMemcpyAsync(ws.inputs.p, h, bt->inputs_bytes, cudaMemcpyHostToDevice, st)
             : cudaMemcpy(ws.inputs.p, h, bt->inputs_bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e);
  // Test switch: fill the boundary records and slab planes with 0x3F3F3F3F, a value far above
  // any score, so that a kernel reading a record slot before (or without) its producer writing
  // it gives a wrong result instead of one that fresh, zeroed memory would hide.
  if (bt->plan->test_poison) {
    if (ws.faces.p && (e = cudaMemsetAsync(ws.faces.p, 0x3F, ws.faces.cap, st)) != cudaSuccess)
      return cuda_status(e);
    if (ws.planes.p && (e = cudaMemsetAsync(ws.planes.p, 0x3F, ws.planes.cap, st)) != cudaSuccess)
      return cuda_status(e);
  }
  bt->uploaded = true;
  bt->h2d_bytes = bt->inputs_bytes;
  return TRIOSEQ_OK;
}

// Event record that also works inside a stream capture (there it becomes an event-record node
// instead of a capture-internal dependency).
cudaError_t record(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  return cudaEventRecord(ev, st);
}

// One pass of the hot path on device-resident inputs.
trioseq_status run(trioseq_batch_s* bt, cudaStream_t st) {
  Workspace& ws = *bt->ws;
  trioseq_plan_s* plan = bt->plan;
  const bool tb = bt->mode == TRIOSEQ_WITH_TRACEBACK;
  const size_t nprog = bt->tasks.size() + 64;
  int32_t* prog = ws.progress.as<int32_t>();
  int32_t* queue = prog + bt->tasks.size();
  int32_t* err = queue + 32;
  cudaError_t e = cudaMemsetAsync(prog, 0, nprog * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_status(e);
  if (bt->n == 0) return TRIOSEQ_OK;
  char* in = ws.inputs.as<char>();
  if (plan->affine) {  // affine gaps (affine.cu): score only, one CTA per triplet at a time
    AffineParams ap{};
    ap.desc = reinterpret_cast<const TripDesc*>(in + bt->off_desc);
    ap.tasks = reinterpret_cast<const Task*>(in + bt->off_tasks);
    ap.n = (int32_t)bt->tasks.size();
    ap.KP = plan->KP;
    ap.seq = reinterpret_cast<const int8_t*>(in);
    ap.sub = plan->sig_affine.as<int32_t>();
    ap.gap = plan->gap;
    ap.gap_open = plan->gap_open;
    ap.planes = ws.faces.as<int32_t>();
    ap.plane_cells = bt->affine_cells;
    ap.queue = queue;
    ap.scores = ws.scores.as<int32_t>();
    if (bt->profile && record(bt->ev[0], st) != cudaSuccess) return cuda_status(cudaGetLastError());
    if (launch_affine(ap, bt->grid, st) != 0) return cuda_status(cudaGetLastError());
    if (bt->profile) {
      if (record(bt->ev[1], st) != cudaSuccess || record(bt->ev[2], st) != cudaSuccess)
        return cuda_status(cudaGetLastError());
      bt->timed = true;
    }
    return TRIOSEQ_OK;
  }
  WaveParams p{};
  p.desc = reinterpret_cast<const TripDesc*>(in + bt->off_desc);
  p.tasks = reinterpret_cast<const Task*>(in + bt->off_tasks);
  p.ntasks = (int32_t)bt->tasks.size();
  p.KP = plan->KP;
  p.seq = reinterpret_cast<const int8_t*>(in);
  p.sig = tb ? plan->sig_tb.as<int32_t>() : plan->sig_score.as<int32_t>();
  p.faces = ws.faces.as<int32_t>();
  p.progress = prog;
  p.queue = queue;
  p.codes = tb ? ws.codes.as<uint32_t>() : nullptr;
  p.scores = ws.scores.as<int32_t>();
  p.err = err;
  p.TI = std::max(1, bt->TI);
  p.wait_ns = plan->wait_ns;
  p.g2 = -2 * plan->gap;
  p.one = 1;
  // One-triplet traceback launches, whose time is the wavefront ramp: records carry their own
  // readiness (sentinel-filled here, in the launch's stream order), so each producer-consumer
  // level lags by its skew alone instead of also by a publication interval and a flag round
  // trip; progress is then published only at the end of a task. TRIOSEQ_DATA_FLAGS at plan
  // creation forces it on (1) or off (0) for every traceback launch.
  p.data_flags = tb && !bt->slab && (plan->data_flags >= 0 ? plan->data_flags : bt->n == 1);
  if (p.data_flags) {
    if ((e = cudaMemsetAsync(p.faces, 0x80, bt->face_ints * sizeof(int32_t), st)) != cudaSuccess)
      return cuda_status(e);
    p.TI = 1 << 30;
  }
  const int warps_per_cta = wavefront_block_threads(bt->packed) / 32;  // resident warps per CTA
  if (plan->test_wait_unset && !bt->slab) {
    // Test of the bounded waits: every first-wave task but queue task 0 waits on a word of the
    // progress buffer that nothing writes (zeroed above), gives up after wait_ns, sets the error
    // word and returns; the call then reports TRIOSEQ_ETIMEOUT.
    p.pace_n = bt->grid * warps_per_cta;
    p.pace_T = 1 << 20;
    p.pace_flag = prog + bt->tasks.size() + 48;
  } else if (!bt->slab && plan->pace && !p.data_flags &&
             bt->tasks.size() >= 2 * (size_t)bt->grid * warps_per_cta) {
    // pace the first wave against the progress of queue task 0, the (0,0) block of its triplet
    const TripDesc& d0 = bt->desc[bt->tasks[0].trip];
    p.pace_n = bt->grid * warps_per_cta;
    p.pace_T = d0.T;
    p.pace_flag = prog + d0.prog_base;
  }
  if (tb && plan->atype != kGlobal) {  // (score, first cell) keys start from 0
    p.best64 = ws.best64.as<unsigned long long>();
    if ((e = cudaMemsetAsync(p.best64, 0, bt->n * sizeof(unsigned long long), st)) != cudaSuccess)
      return cuda_status(e);
  }
  // Semi-global and local scores are maxima accumulated with atomicMax: start from 0x80808080.
  if (plan->atype != kGlobal &&
      (e = cudaMemsetAsync(p.scores, 0x80, bt->n * sizeof(int32_t), st)) != cudaSuccess)
    return cuda_status(e);
  WalkParams w{};
  w.desc = p.desc;
  w.tb_trips = reinterpret_cast<const int32_t*>(in + bt->off_tb);
  w.ntb = (int32_t)bt->tb_trips.size();
  w.seq = p.seq;
  w.codes = p.codes;
  w.rows = ws.rows.as<uint8_t>();
  w.row_off = reinterpret_cast<const int64_t*>(in + bt->off_rowoff);
  w.row_cap = reinterpret_cast<const int32_t*>(in + bt->off_rowcap);
  w.aln_len = ws.lens.as<int32_t>();
  w.err = err;
  w.NJ = bt->var.nj;
  w.NK = bt->var.nk;
  w.atype = plan->atype;
  w.best64 = p.best64;
  w.scores = p.scores;
  w.span = tb ? ws.spans.as<int32_t>() : nullptr;
  bt->timed = false;
  if (bt->profile && record(bt->ev[0], st) != cudaSuccess)
    return cuda_status(cudaGetLastError());
  if (bt->slab) {
    // Slab mode. Slab m covers the slices m*S .. of the cube; plane m holds its last slice.
    // Score: forward through all slabs, planes ping-pong. Traceback: forward through all but the
    // top slab keeping every plane (no codes), then from the top slab down: recompute the slab
    // with codes from the plane below it and continue the walk through it.
    const TripDesc* sdesc = reinterpret_cast<const TripDesc*>(in + bt->off_slab);
    int32_t* planes = ws.planes.as<int32_t>();
    const auto plane = [&](int idx) { return planes + (size_t)idx * bt->plane_ints; };
    const auto wave = [&](int m, const int32_t* pin, int32_t* pout, bool codes) {
      const cudaError_t ee = cudaMemsetAsync(prog, 0, nprog * sizeof(int32_t), st);
      if (ee != cudaSuccess) return cuda_status(ee);
      WaveParams q = p;
      q.desc = sdesc + m;
      q.i0 = m * bt->slab;
      q.plane_in = pin;
      q.plane_out = pout;
      q.codes = codes ? p.codes : nullptr;
      if (launch_wavefront(bt->var.nj, bt->var.nk, tb, kGlobal, false, true, q, bt->grid,
                           bt->smem, st) != 0)
        return cuda_status(cudaGetLastError());
      return TRIOSEQ_OK;
    };
    const int M = bt->nslab;
    trioseq_status s = TRIOSEQ_OK;
    if (!tb) {
      for (int m = 0; m < M && s == TRIOSEQ_OK; m++)
        s = wave(m, m ? plane((m - 1) & 1) : nullptr, m + 1 < M ? plane(m & 1) : nullptr, false);
    } else {
      for (int m = 0; m + 1 < M && s == TRIOSEQ_OK; m++)
        s = wave(m, m ? plane(m - 1) : nullptr, plane(m), false);
      for (int m = M - 1; m >= 0 && s == TRIOSEQ_OK; m--) {
        s = wave(m, m ? plane(m - 1) : nullptr, nullptr, true);
        if (s != TRIOSEQ_OK) break;
        WalkParams wm = w;
        wm.i_lo = m * bt->slab;
        wm.T_slab = bt->slab_desc[m].T;  // steps per task of the slab that wrote the codes
        wm.state = ws.walkstate.as<int32_t>();
        wm.init_state = (m == M - 1) ? 1 : 0;
        if (launch_walk(wm, st) != 0) s = cuda_status(cudaGetLastError());
      }
    }
    if (s != TRIOSEQ_OK) return s;
    if (bt->profile && record(bt->ev[1], st) != cudaSuccess)
      return cuda_status(cudaGetLastError());
  } else {
    if (launch_wavefront(bt->var.nj, bt->var.nk, tb, plan->atype, bt->packed, false, p, bt->grid,
                         bt->smem, st) != 0)
      return cuda_status(cudaGetLastError());
    if (bt->profile && record(bt->ev[1], st) != cudaSuccess)
      return cuda_status(cudaGetLastError());
    if (tb && !bt->tb_trips.empty() && launch_walk(w, st) != 0)
      return cuda_status(cudaGetLastError());
  }
  if (bt->profile) {
    if (record(bt->ev[2], st) != cudaSuccess) return cuda_status(cudaGetLastError());
    bt->timed = true;
  }
  return TRIOSEQ_OK;
}

// trioseq_batch_run: replay the batch's graph, capturing it first (on a private stream, so the
// caller's stream may be the legacy default stream) when there is none yet or the workspace
// buffers or the profiling switch changed since it was captured.
trioseq_status run_graph(trioseq_batch_s* bt, cudaStream_t st) {
  const Workspace& ws = *bt->ws;
  // every device address a captured launch bakes in (the slab and walk launches included)
  const std::array<const void*, 12> key{ws.inputs.p,    ws.faces.p,     ws.progress.p,
                                        ws.codes.p,     ws.scores.p,    ws.rows.p,
                                        ws.lens.p,      ws.planes.p,    ws.walkstate.p,
                                        ws.best64.p,    ws.spans.p,
                                        bt->profile ? (const void*)bt->ev[0] : nullptr};
  if (!bt->gexec || key != bt->gkey) {
    if (bt->gexec) {
      cudaGraphExecDestroy(bt->gexec);
      bt->gexec = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!bt->capture_stream)
      e = cudaStreamCreateWithFlags(&bt->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaStreamBeginCapture(bt->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_status(e);
    const trioseq_status s = run(bt, bt->capture_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(bt->capture_stream, &graph);
    if (s == TRIOSEQ_OK && e == cudaSuccess) e = cudaGraphInstantiate(&bt->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (s != TRIOSEQ_OK) return s;
    if (e != cudaSuccess) {
      bt->gexec = nullptr;
      return cuda_status(e);
    }
    bt->gkey = key;
  }
  bt->timed = false;
  const cudaError_t e = cudaGraphLaunch(bt->gexec, st);
  if (e != cudaSuccess) return cuda_status(e);
  bt->timed = bt->profile;
  return TRIOSEQ_OK;
}

// Wait for the run, check the error word, fetch scores (and traceback rows).
trioseq_status fetch(trioseq_batch_s* bt, cudaStream_t st, int32_t* scores_out) {
  Workspace& ws = *bt->ws;
  const bool tb = bt->mode == TRIOSEQ_WITH_TRACEBACK;
  int32_t herr = 0;
  cudaError_t e = cudaSuccess;
  if (bt->n) {
    int32_t* err = ws.progress.as<int32_t>() + bt->tasks.size() + 32;
    e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && scores_out)
      e = cudaMemcpyAsync(scores_out, ws.scores.p, bt->n * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && tb && !bt->tb_trips.empty()) {
      bt->h_rows.resize(bt->rows_bytes);
      bt->h_lens.resize(bt->tb_trips.size());
      e = cudaMemcpyAsync(bt->h_rows.data(), ws.rows.p, bt->rows_bytes, cudaMemcpyDeviceToHost,
                          st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(bt->h_lens.data(), ws.lens.p, bt->h_lens.size() * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st);
      bt->h_spans.resize(6 * bt->tb_trips.size());
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(bt->h_spans.data(), ws.spans.p, bt->h_spans.size() * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  if (herr & 1) return TRIOSEQ_ETIMEOUT;
  if (herr & 2) return TRIOSEQ_ECUDA;
  bt->have_rows = tb;
  bt->d2h_bytes = bt->n ? sizeof(int32_t) * (1 + bt->n) : 0;
  if (tb && !bt->tb_trips.empty())
    bt->d2h_bytes += bt->rows_bytes + bt->h_lens.size() * sizeof(int32_t) +
                     bt->h_spans.size() * sizeof(int32_t);
  return TRIOSEQ_OK;
}

trioseq_status copy_span(const trioseq_batch_s* bt, size_t idx, int32_t* begin, int32_t* end) {
  if (!bt || !bt->have_rows || idx >= bt->n || !begin || !end) return TRIOSEQ_EINVAL;
  const int32_t q = bt->tb_of[idx];
  if (q < 0 || bt->h_lens[q] < 0) return TRIOSEQ_EINVAL;
  for (int t = 0; t < 3; t++) {
    begin[t] = bt->h_spans[6 * q + t];
    end[t] = bt->h_spans[6 * q + 3 + t];
  }
  return TRIOSEQ_OK;
}

trioseq_status copy_alignment(const trioseq_batch_s* bt, size_t idx, char* r0, char* r1, char* r2,
                              size_t cap, size_t* aln_len) {
  if (!bt || !bt->have_rows || idx >= bt->n || !aln_len) return TRIOSEQ_EINVAL;
  const int32_t q = bt->tb_of[idx];
  if (q < 0) return TRIOSEQ_EINVAL;
  const int32_t L = bt->h_lens[q];
  if (L < 0) return TRIOSEQ_ECUDA;
  *aln_len = (size_t)L;
  if (L == 0) return TRIOSEQ_OK;
  if (cap < (size_t)L || !r0 || !r1 || !r2) return TRIOSEQ_EINVAL;
  const int32_t rc = bt->row_cap[q];
  const uint8_t* base = bt->h_rows.data() + bt->row_off[q];
  const char* alpha = bt->plan->alphabet;
  char* out[3] = {r0, r1, r2};
  for (int s = 0; s < 3; s++) {
    const uint8_t* row = base + (size_t)s * rc + (rc - L);
    for (int32_t t = 0; t < L; t++) out[s][t] = row[t] == 255 ? '-' : alpha[row[t]];
  }
  return TRIOSEQ_OK;
}

}  // namespace

extern "C" {

const char* trioseq_strerror(trioseq_status st) {
  switch (st) {
    case TRIOSEQ_OK: return "ok";
    case TRIOSEQ_EINVAL: return "invalid argument";
    case TRIOSEQ_ENOMEM: return "out of memory";
    case TRIOSEQ_EAGAIN: return "not ready / queue full";
    case TRIOSEQ_EOVERFLOW: return "score bound exceeds the integer range";
    case TRIOSEQ_ETIMEOUT: return "bounded device wait expired";
    case TRIOSEQ_ECUDA: return "CUDA error or no usable GPU";
    case TRIOSEQ_ENOTIMPL: return "not implemented";
    case TRIOSEQ_ESCRATCH: return "request exceeds the fixed scratch of the allocation-free call";
  }
  return "unknown status";
}

trioseq_status trioseq_plan(const trioseq_scoring* sc, uint32_t max_len_hint, uint32_t flags,
                            trioseq_plan_t* out) {
  return no_throw([&]() -> trioseq_status {
    (void)max_len_hint;
    NvtxRange range("trioseq_plan");
    if (!out) return TRIOSEQ_EINVAL;
    *out = nullptr;
    if (!sc || !sc->alphabet || !sc->sub || flags > TRIOSEQ_LOCAL) return TRIOSEQ_EINVAL;
    const int K = sc->alphabet_size;
    if (K < 1 || K > kMaxAlphabet || sc->gap > 0 || sc->gap < -127) return TRIOSEQ_EINVAL;
    std::unique_ptr<trioseq_plan_s> plan(new (std::nothrow) trioseq_plan_s());
    if (!plan) return TRIOSEQ_ENOMEM;
    for (int i = 0; i < 256; i++) plan->lut[i] = -1;
    for (int i = 0; i < K; i++) {
      const unsigned char ch = (unsigned char)sc->alphabet[i];
      if (plan->lut[ch] >= 0) return TRIOSEQ_EINVAL;  // duplicate residue
      plan->lut[ch] = (int16_t)i;
      plan->alphabet[i] = (char)ch;
    }
    for (int i = 0; i < K; i++)
      for (int j = 0; j < K; j++)
        if (sc->sub[i * K + j] != sc->sub[j * K + i]) return TRIOSEQ_EINVAL;
    plan->K = K;
    plan->KP = K + 1;
    plan->gap = sc->gap;
    plan->atype = (int)flags;
    plan->sub.assign(sc->sub, sc->sub + K * K);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      return TRIOSEQ_ECUDA;
    }
    plan->device = dev;
    if (cudaDeviceGetAttribute(&plan->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return TRIOSEQ_ECUDA;
    }
    const int KP = K + 1;
    std::vector<int32_t> s2((size_t)KP * KP, 0), s8((size_t)KP * KP, 0);
    int32_t mx = 0, mn = 0;
    for (int i = 0; i < K; i++)
      for (int j = 0; j < K; j++) {
        const int32_t v = (int32_t)sc->sub[i * K + j] - 2 * sc->gap;  // sigma'' = sigma - 2 alpha
        s2[(size_t)i * KP + j] = v;
        s8[(size_t)i * KP + j] = 8 * v;
        mx = std::max(mx, std::abs(v));
        mn = std::min(mn, v);
      }
    plan->max_abs_sig2 = std::max(mx, 1);
    plan->sig2_nonneg = mn >= 0;
    // The plan's device memory is allocated and freed in the order of its own stream.
    if (plan->ws.make_own_stream() != cudaSuccess) return cuda_status(cudaGetLastError());
    cudaStream_t as = plan->ws.alloc_stream;
    if (!plan->sig_score.ensure(s2.size() * 4, as) || !plan->sig_tb.ensure(s8.size() * 4, as))
      return TRIOSEQ_ENOMEM;
    if (cudaMemcpyAsync(plan->sig_score.p, s2.data(), s2.size() * 4, cudaMemcpyHostToDevice,
                        as) != cudaSuccess ||
        cudaMemcpyAsync(plan->sig_tb.p, s8.data(), s8.size() * 4, cudaMemcpyHostToDevice, as) !=
            cudaSuccess ||
        cudaStreamSynchronize(as) != cudaSuccess)
      return cuda_status(cudaGetLastError());
    plan->TI = std::max(1, env_int("TRIOSEQ_TI", 8));
    plan->graphs = env_int("TRIOSEQ_GRAPHS", 1) != 0;
    plan->packed16 = env_int("TRIOSEQ_PACKED", 1) != 0;
    plan->pace = env_int("TRIOSEQ_PACE", 1) != 0;
    plan->wait_ns = (int64_t)std::max(1, env_int("TRIOSEQ_WAIT_MS", 2000)) * 1000000LL;
    plan->test_wait_unset = env_int("TRIOSEQ_TEST_WAIT_UNSET", 0) != 0;
    plan->test_poison = env_int("TRIOSEQ_TEST_POISON", 0) != 0;
    plan->data_flags = env_int("TRIOSEQ_DATA_FLAGS", -1);
    g_alloc_calls.store(0);
    g_alloc_fail_at.store(std::max(0, env_int("TRIOSEQ_TEST_FAIL_ALLOC", 0)));
    {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
      }
      const int mb = env_int("TRIOSEQ_SLAB_BUDGET_MB", 0);
      plan->slab_budget = mb > 0 ? (size_t)mb << 20 : fr / 2;
      plan->slab_slices = std::max(0, env_int("TRIOSEQ_SLAB_SLICES", 0));
    }
    // "RxC": register tile rows x columns per lane
    const auto parse_tile = [](const char* v, Variant* out) {
      if (!v) return;
      char* end = nullptr;
      const long rj = std::strtol(v, &end, 10);
      if (!end || *end != 'x') return;
      char* end2 = nullptr;
      const long ck = std::strtol(end + 1, &end2, 10);
      // "8x16" and a trailing 'v' ("8x8v") select the two-cells-per-register kernel; a trailing
      // 's' or 't' ("8x16s", "8x16t") its variants with the sigma''(y,z) tile in shared memory
      const char sfx = end2 ? *end2 : 0;
      const int two = sfx == 's' ? 2 : (sfx == 't' ? 3 : ((ck == 16 || sfx == 'v') ? 1 : 0));
      if (rj > 0 && rj <= 16 && ck > 0 && ck <= 32) *out = Variant{(int)rj, (int)ck, two};
    };
    parse_tile(std::getenv("TRIOSEQ_SCORE_TILE"), &plan->score_variant);
    parse_tile(std::getenv("TRIOSEQ_TB_TILE"), &plan->tb_variant);
    *out = plan.release();
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_plan_affine(const trioseq_scoring* sc, int32_t gap_open, uint32_t flags,
                                   trioseq_plan_t* out) {
  return no_throw([&]() -> trioseq_status {
    NvtxRange range("trioseq_plan_affine");
    if (!out) return TRIOSEQ_EINVAL;
    *out = nullptr;
    if (flags != TRIOSEQ_GLOBAL || gap_open > 0 || gap_open < -(1 << 20)) return TRIOSEQ_EINVAL;
    trioseq_plan_t plan = nullptr;
    trioseq_status s = trioseq_plan(sc, 0, flags, &plan);
    if (s != TRIOSEQ_OK) return s;
    std::unique_ptr<trioseq_plan_s, trioseq_status (*)(trioseq_plan_t)> keep(
        plan, &trioseq_plan_destroy);
    DeviceGuard g(plan->device);
    plan->affine = true;
    plan->gap_open = gap_open;
    const int K = plan->K, KP = plan->KP;
    std::vector<int32_t> tab((size_t)KP * KP, 0);
    int32_t mx = 0;
    for (int i = 0; i < K; i++)
      for (int j = 0; j < K; j++) {
        tab[(size_t)i * KP + j] = sc->sub[i * K + j];
        mx = std::max(mx, std::abs((int32_t)sc->sub[i * K + j]));
      }
    plan->max_abs_sub = mx;
    cudaStream_t as = plan->ws.alloc_stream;
    if (!plan->sig_affine.ensure(tab.size() * 4, as)) return TRIOSEQ_ENOMEM;
    if (cudaMemcpyAsync(plan->sig_affine.p, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice,
                        as) != cudaSuccess ||
        cudaStreamSynchronize(as) != cudaSuccess)
      return cuda_status(cudaGetLastError());
    *out = keep.release();
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_plan_destroy(trioseq_plan_t plan) {
  return no_throw([&]() -> trioseq_status {
    if (!plan) return TRIOSEQ_OK;
    DeviceGuard g(plan->device);
    // Wait for the plan's own last use only (its trioseq_align_batch work); batches made from
    // the plan are destroyed before it and have waited for theirs. Other streams, a running
    // server's included, are not synchronised. The substitution tables are freed in the order
    // of the plan's stream, before the workspace releases that stream.
    plan->ws.wait_last_use();
    plan->last.reset();
    plan->ws.order_after_last_use();
    plan->sig_score.reset();
    plan->sig_tb.reset();
    plan->sig_affine.reset();
    delete plan;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_align_batch(trioseq_plan_t plan, const trioseq_triplet* triplets, size_t n,
                                   uint32_t mode, int32_t* scores_out, void* stream) {
  return no_throw([&]() -> trioseq_status {
    NvtxRange range("trioseq_align_batch");
    if (!plan || (n && !scores_out)) return TRIOSEQ_EINVAL;
    DeviceGuard g(plan->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_ptr<trioseq_batch_s> bt(new (std::nothrow) trioseq_batch_s());
    if (!bt) return TRIOSEQ_ENOMEM;
    plan->last.reset();
    trioseq_status s = build_batch(plan, triplets, n, mode, bt.get());
    if (s != TRIOSEQ_OK) return s;
    bt->ws = &plan->ws;
    if ((s = upload(bt.get(), st, true)) != TRIOSEQ_OK) return s;
    s = run(bt.get(), st);
    plan->ws.mark_use(st);  // also after a partial enqueue: destroy waits for what did run
    if (s != TRIOSEQ_OK) return s;
    if ((s = fetch(bt.get(), st, scores_out)) != TRIOSEQ_OK) return s;
    bt->seq.clear();
    bt->seq.shrink_to_fit();
    plan->last = std::move(bt);
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_traceback(trioseq_plan_t plan, size_t idx, char* row0, char* row1,
                                 char* row2, size_t cap, size_t* aln_len) {
  return no_throw([&]() -> trioseq_status {
    NvtxRange range("trioseq_traceback");
    if (!plan || !plan->last) return TRIOSEQ_EINVAL;
    return copy_alignment(plan->last.get(), idx, row0, row1, row2, cap, aln_len);
  });
}

trioseq_status trioseq_traceback_span(trioseq_plan_t plan, size_t idx, int32_t begin[3],
                                      int32_t end[3]) {
  return no_throw([&]() -> trioseq_status {
    if (!plan || !plan->last) return TRIOSEQ_EINVAL;
    return copy_span(plan->last.get(), idx, begin, end);
  });
}

trioseq_status trioseq_batch_create(trioseq_plan_t plan, const trioseq_triplet* triplets,
                                    size_t n, uint32_t mode, trioseq_batch_t* out) {
  return no_throw([&]() -> trioseq_status {
    NvtxRange range("trioseq_batch_create");
    if (!plan || !out) return TRIOSEQ_EINVAL;
    *out = nullptr;
    DeviceGuard g(plan->device);
    std::unique_ptr<trioseq_batch_s> bt(new (std::nothrow) trioseq_batch_s());
    if (!bt) return TRIOSEQ_ENOMEM;
    trioseq_status s = build_batch(plan, triplets, n, mode, bt.get());
    if (s != TRIOSEQ_OK) return s;
    bt->own_ws.reset(new (std::nothrow) Workspace());
    if (!bt->own_ws) return TRIOSEQ_ENOMEM;
    if (bt->own_ws->make_own_stream() != cudaSuccess) return cuda_status(cudaGetLastError());
    bt->ws = bt->own_ws.get();
    if ((s = upload(bt.get(), nullptr, false)) != TRIOSEQ_OK) return s;
    *out = bt.release();
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_run(trioseq_batch_t bt, void* stream) {
  return no_throw([&]() -> trioseq_status {
    NvtxRange range("trioseq_batch_run");
    if (!bt) return TRIOSEQ_EINVAL;
    DeviceGuard g(bt->plan->device);
    const cudaStream_t st = (cudaStream_t)stream;
    const trioseq_status s = bt->plan->graphs ? run_graph(bt, st) : run(bt, st);
    const cudaError_t e = bt->ws->mark_use(st);
    return s != TRIOSEQ_OK ? s : cuda_status(e);
  });
}

trioseq_status trioseq_batch_scores(trioseq_batch_t bt, void* stream, int32_t* scores_out) {
  return no_throw([&]() -> trioseq_status {
    if (!bt || (bt->n && !scores_out)) return TRIOSEQ_EINVAL;
    DeviceGuard g(bt->plan->device);
    return fetch(bt, (cudaStream_t)stream, scores_out);
  });
}

trioseq_status trioseq_batch_device_scores(trioseq_batch_t bt, int32_t** d_scores) {
  return no_throw([&]() -> trioseq_status {
    if (!bt || !d_scores) return TRIOSEQ_EINVAL;
    *d_scores = bt->ws->scores.as<int32_t>();
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_alignment(trioseq_batch_t bt, size_t idx, char* row0, char* row1,
                                       char* row2, size_t cap, size_t* aln_len) {
  return no_throw([&]() -> trioseq_status {
    return copy_alignment(bt, idx, row0, row1, row2, cap, aln_len);
  });
}

trioseq_status trioseq_batch_span(trioseq_batch_t bt, size_t idx, int32_t begin[3],
                                  int32_t end[3]) {
  return no_throw([&]() -> trioseq_status {
    return copy_span(bt, idx, begin, end);
  });
}

trioseq_status trioseq_batch_info(trioseq_batch_t bt, size_t* n, uint64_t* cells, uint64_t* tasks,
                                  int32_t* tile_j, int32_t* tile_k) {
  return no_throw([&]() -> trioseq_status {
    if (!bt) return TRIOSEQ_EINVAL;
    if (n) *n = bt->n;
    if (cells) *cells = bt->cells;
    if (tasks) *tasks = bt->tasks.size();
    if (tile_j) *tile_j = bt->var.nj;
    if (tile_k) *tile_k = bt->var.nk;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_slabs(trioseq_batch_t bt, int32_t* slices, int32_t* slabs) {
  return no_throw([&]() -> trioseq_status {
    if (!bt || !slices || !slabs) return TRIOSEQ_EINVAL;
    *slices = bt->slab;
    *slabs = bt->nslab;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_packing(trioseq_batch_t bt, int32_t* per_word) {
  return no_throw([&]() -> trioseq_status {
    if (!bt || !per_word) return TRIOSEQ_EINVAL;
    *per_word = bt->packed ? 2 : 1;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_kernel(trioseq_batch_t bt, char* name, size_t cap) {
  return no_throw([&]() -> trioseq_status {
    if (!bt || !name || cap == 0) return TRIOSEQ_EINVAL;
    const bool tb = bt->mode == TRIOSEQ_WITH_TRACEBACK;
    const int at = bt->plan->atype;
    const char* type = at == kLocal ? "local" : (at == kSemiGlobal ? "semiglobal" : "global");
    const int nj = bt->var.nj, nk = bt->var.nk;
    char buf[160];
    if (bt->plan->affine)
      std::snprintf(buf, sizeof buf, "affine_kernel tile plane");
    else if (bt->packed >= 3)
      std::snprintf(buf, sizeof buf, "wavefront_vl_kernel<%d,%d,%d> tile %dx%d%s", nj, nk / 2,
                    bt->packed - 3, nj, nk,
                    bt->packed == 4 ? "s" : (bt->packed == 5 ? "t" : (nk == 16 ? "" : "v")));
    else if (bt->packed)
      std::snprintf(buf, sizeof buf, "wavefront_kernel<%d,%d,score,global,%s> tile %dx%d", nj, nk,
                    bt->packed == 2 ? "two triplets per register, biased" :
                                      "two triplets per register, signed", nj, nk);
    else
      std::snprintf(buf, sizeof buf, "wavefront_kernel<%d,%d,%s,%s%s> tile %dx%d", nj, nk,
                    tb ? "traceback" : "score", type, bt->slab ? ",slab" : "", nj, nk);
    std::snprintf(name, cap, "%s", buf);
    return std::strlen(buf) < cap ? TRIOSEQ_OK : TRIOSEQ_EINVAL;
  });
}

trioseq_status trioseq_batch_profile(trioseq_batch_t bt, int32_t enable) {
  return no_throw([&]() -> trioseq_status {
    if (!bt) return TRIOSEQ_EINVAL;
    DeviceGuard g(bt->plan->device);
    if (enable)
      for (auto& e : bt->ev)
        if (!e && cudaEventCreate(&e) != cudaSuccess) return cuda_status(cudaGetLastError());
    bt->profile = enable != 0;
    bt->timed = false;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_timing(trioseq_batch_t bt, float ms[2]) {
  return no_throw([&]() -> trioseq_status {
    if (!bt || !ms || !bt->profile || !bt->timed) return TRIOSEQ_EINVAL;
    DeviceGuard g(bt->plan->device);
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, bt->ev[0], bt->ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, bt->ev[1], bt->ev[2]) != cudaSuccess)
      return cuda_status(cudaGetLastError());
    ms[0] = a;
    ms[1] = b;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_plan_autotune(trioseq_plan_t plan, const trioseq_triplet* sample, size_t n,
                                     uint32_t mode, int32_t* tile_j, int32_t* tile_k,
                                     int32_t* ti) {
  return no_throw([&]() -> trioseq_status {
    NvtxRange range("trioseq_plan_autotune");
    if (!plan || !sample || n == 0 || mode > TRIOSEQ_WITH_TRACEBACK) return TRIOSEQ_EINVAL;
    DeviceGuard g(plan->device);
    if (plan->affine) {  // one kernel shape: nothing to choose
      if (tile_j) *tile_j = 0;
      if (tile_k) *tile_k = 0;
      if (ti) *ti = 0;
      return mode == TRIOSEQ_WITH_TRACEBACK ? TRIOSEQ_ENOTIMPL : TRIOSEQ_OK;
    }
    // candidate tiles per mode; 8x4 exists for traceback keys only
    // 8x16 and 8x8 with vl: two cells of one triplet per register
    static const Variant kScoreTiles[] = {{8, 8},    {4, 8},    {4, 4},   {8, 16, 1},
                                          {8, 8, 1}, {8, 16, 2}, {8, 16, 3}};
    static const Variant kTbTiles[] = {{8, 8}, {4, 8}, {4, 4}, {8, 4}};
    static const int kTI[] = {4, 8, 16, 32};
    const bool tb_mode = mode == TRIOSEQ_WITH_TRACEBACK;
    const Variant* tiles = tb_mode ? kTbTiles : kScoreTiles;
    const size_t ntiles = tb_mode ? sizeof(kTbTiles) / sizeof(kTbTiles[0])
                                  : sizeof(kScoreTiles) / sizeof(kScoreTiles[0]);
    uint32_t maxlen = 0;
    for (size_t t = 0; t < n; t++)
      for (int q = 0; q < 3; q++) maxlen = std::max(maxlen, sample[t].len[q]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return cuda_status(cudaGetLastError());
    trioseq_status result = TRIOSEQ_OK;
    float best = 3.0e38f;
    trioseq_plan_s::Tuned bestv{mode == TRIOSEQ_WITH_TRACEBACK ? plan->tb_variant
                                                               : plan->score_variant,
                                plan->TI};
    {
      Workspace ws;  // one workspace, grown to the largest candidate
      plan->tuning = true;
      for (size_t vi = 0; vi < ntiles; vi++) {
        const Variant& v = tiles[vi];
        for (int ti : kTI) {
          plan->forced = trioseq_plan_s::Tuned{v, ti};
          trioseq_batch_s bt;
          trioseq_status s = build_batch(plan, sample, n, mode, &bt);
          if (s == TRIOSEQ_ECUDA) continue;  // variant cannot be resident with this alphabet
          if (s != TRIOSEQ_OK) {
            result = s;
            break;
          }
          bt.ws = &ws;
          if ((s = upload(&bt, nullptr, false)) != TRIOSEQ_OK ||
              (s = run(&bt, nullptr)) != TRIOSEQ_OK ||
              (s = fetch(&bt, nullptr, nullptr)) != TRIOSEQ_OK) {
            result = s;
            break;
          }
          float ms = 0.f;
          cudaEventRecord(e0, nullptr);
          for (int rep = 0; rep < 2 && s == TRIOSEQ_OK; rep++) s = run(&bt, nullptr);
          cudaEventRecord(e1, nullptr);
          if (s == TRIOSEQ_OK) s = fetch(&bt, nullptr, nullptr);
          if (s != TRIOSEQ_OK || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            result = s != TRIOSEQ_OK ? s : cuda_status(cudaGetLastError());
            break;
          }
          if (ms < best) {
            best = ms;
            bestv = trioseq_plan_s::Tuned{v, ti};
          }
        }
        if (result != TRIOSEQ_OK) break;
      }
      plan->tuning = false;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != TRIOSEQ_OK) return result;
    plan->tuned[tune_key(mode, n, maxlen)] = bestv;
    if (tile_j) *tile_j = bestv.var.nj;
    if (tile_k) *tile_k = bestv.var.nk;
    if (ti) *ti = bestv.TI;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_plan_io_bytes(trioseq_plan_t plan, uint64_t* h2d, uint64_t* d2h) {
  return no_throw([&]() -> trioseq_status {
    if (!plan || !plan->last) return TRIOSEQ_EINVAL;
    if (h2d) *h2d = plan->last->h2d_bytes;
    if (d2h) *d2h = plan->last->d2h_bytes;
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_batch_destroy(trioseq_batch_t bt) {
  return no_throw([&]() -> trioseq_status {
    if (!bt) return TRIOSEQ_OK;
    DeviceGuard g(bt->plan->device);
    // Wait for this batch's own last run only; its buffers are then freed in the order of its
    // private stream. Other streams (a running server's included) are not synchronised.
    bt->ws->wait_last_use();
    delete bt;
    return TRIOSEQ_OK;
  });
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Serving: continuous batching behind submit/poll.
//
// A server thread owns a FIFO of requests and kSlots slots, each a CUDA stream with its own
// reusable workspace and pinned result buffer. Every tick it (1) harvests slots whose launch has
// completed (event query, never a blocking wait) and publishes their results, then (2) admits
// pending requests into free slots: the oldest request fixes the (scoring, mode) group, and
// further requests of that group join the launch in arrival order while the launch's workspace
// estimate stays within the slot's share of the device-memory budget. Requests that arrive
// while other launches run are therefore admitted as soon as a slot frees, and launches of
// different slots overlap on the device. poll() only looks up the result table.
namespace {

using Clock = std::chrono::steady_clock;

struct SrvReq {
  uint64_t ticket = 0;
  int32_t plan_id = 0;
  uint32_t mode = 0;
  std::string s[3];
  size_t bytes = 0;        // workspace estimate inside a launch of several requests
  size_t bytes_alone = 0;  // estimate of a launch of this request alone (slab form if it applies)
};

struct SrvRes {
  trioseq_status st = TRIOSEQ_OK;
  int32_t score = 0;
  bool has_rows = false;
  std::string rows[3];
};

struct SrvSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  Workspace ws;
  HostPinned out;  // scores | error word | alignment lengths | rows
  size_t off_err = 0, off_lens = 0, off_rows = 0;
  std::unique_ptr<trioseq_batch_s> batch;
  std::vector<SrvReq> reqs;
  size_t bytes = 0;  // workspace estimate admitted for the launch on this slot
  trioseq_status launch_st = TRIOSEQ_OK;
};

// Device bytes one request adds to a launch's workspace (boundary records, flags, and in
// traceback mode the code stream and rows).
size_t request_bytes(const trioseq_plan_s* plan, uint32_t mode, const uint32_t len[3]) {
  const bool tb = mode == TRIOSEQ_WITH_TRACEBACK;
  const Variant v = tb ? plan->tb_variant : plan->score_variant;
  const size_t WJ = (size_t)kPR * v.nj, WK = (size_t)kPC * v.nk, W = (size_t)v.nj * v.nk / 8;
  const size_t a = len[0], b = len[1], c = len[2];
  const size_t nJ = (b + 1 + WJ - 1) / WJ, nK = (c + 1 + WK - 1) / WK, T = a + 1 + 10;
  size_t bytes = 4 * nJ * nK * (a + 1) * ((WK + 4) + WJ) + 4 * nJ * nK + 256 + a + b + c + 48;
  if (tb) bytes += 4 * nJ * nK * T * 32 * W + 3 * (a + b + c) + 64;
  return bytes;
}

// The same request launched alone: a global-type triplet whose one-launch workspace exceeds the
// plan's slab budget runs in slabs within that budget (build_batch), so it needs no more.
size_t request_bytes_alone(const trioseq_plan_s* plan, uint32_t mode, const uint32_t len[3]) {
  const size_t full = request_bytes(plan, mode, len);
  return plan->atype == kGlobal ? std::min(full, std::max<size_t>(plan->slab_budget, 1 << 20))
                                : full;
}

size_t workspace_device_bytes(const Workspace& ws) {
  return ws.inputs.cap + ws.faces.cap + ws.progress.cap + ws.codes.cap + ws.scores.cap +
         ws.rows.cap + ws.lens.cap + ws.planes.cap + ws.walkstate.cap + ws.best64.cap +
         ws.spans.cap;
}

}  // namespace

struct trioseq_server_s {
  static constexpr int kSlots = 4;
  std::vector<trioseq_plan_s*> plans;
  int device = 0;
  // Admission by device memory: launches on the device together hold at most `budget` bytes of
  // workspace estimates (in_flight). With no budget given, each admission is also bounded by
  // the memory free on the device at that moment. launch_share (budget / kSlots) caps how many
  // small requests one launch groups, so that several launches overlap; a single larger
  // request may use whatever room is left, and waits for room while other launches run.
  size_t budget = 0;
  size_t launch_share = 0;
  size_t in_flight = 0;
  bool budget_from_free = false;
  size_t max_pending = (size_t)1 << 20;  // TRIOSEQ_SERVER_MAX_PENDING at creation
  size_t max_batch = 1024;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<SrvReq> pending;
  std::unordered_map<uint64_t, SrvRes> done;
  std::unordered_map<uint64_t, int> live;  // submitted and not yet consumed by poll
  uint64_t next_ticket = 1;
  bool stop = false;
  SrvSlot slots[kSlots];
};

namespace {

// Enqueue one launch for the requests in `sl.reqs` on the slot's stream (server thread, no lock).
trioseq_status srv_launch(trioseq_server_s* S, SrvSlot& sl) {
  const int32_t pid = sl.reqs.front().plan_id;
  const uint32_t mode = sl.reqs.front().mode;
  trioseq_plan_s* plan = S->plans[pid];
  std::vector<trioseq_triplet> trips(sl.reqs.size());
  for (size_t i = 0; i < sl.reqs.size(); i++)
    for (int q = 0; q < 3; q++) {
      trips[i].s[q] = sl.reqs[i].s[q].data();
      trips[i].len[q] = (uint32_t)sl.reqs[i].s[q].size();
    }
  sl.batch.reset(new (std::nothrow) trioseq_batch_s());
  if (!sl.batch) return TRIOSEQ_ENOMEM;
  trioseq_batch_s* bt = sl.batch.get();
  trioseq_status st = build_batch(plan, trips.data(), trips.size(), mode, bt);
  if (st != TRIOSEQ_OK) return st;
  bt->ws = &sl.ws;
  if ((st = upload(bt, sl.stream, true)) != TRIOSEQ_OK) return st;
  NvtxRange range("trioseq_server_launch");
  if ((st = run(bt, sl.stream)) != TRIOSEQ_OK) return st;
  const bool tb = mode == TRIOSEQ_WITH_TRACEBACK;
  const size_t n = bt->n, ntb = bt->tb_trips.size();
  sl.off_err = align_up(n * 4, 64);
  sl.off_lens = sl.off_err + 64;
  sl.off_rows = align_up(sl.off_lens + ntb * 4, 64);
  const size_t need = sl.off_rows + (tb ? bt->rows_bytes : 0);
  if (!sl.out.ensure(need)) return TRIOSEQ_ENOMEM;
  char* h = reinterpret_cast<char*>(sl.out.p);
  int32_t* err = sl.ws.progress.as<int32_t>() + bt->tasks.size() + 32;
  cudaError_t e = cudaMemcpyAsync(h, sl.ws.scores.p, n * 4, cudaMemcpyDeviceToHost, sl.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h + sl.off_err, err, 4, cudaMemcpyDeviceToHost, sl.stream);
  if (e == cudaSuccess && tb && ntb) {
    e = cudaMemcpyAsync(h + sl.off_lens, sl.ws.lens.p, ntb * 4, cudaMemcpyDeviceToHost,
                        sl.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h + sl.off_rows, sl.ws.rows.p, bt->rows_bytes, cudaMemcpyDeviceToHost,
                          sl.stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
  return cuda_status(e);
}

// Turn a finished slot into results (server thread, lock held).
void srv_harvest(trioseq_server_s* S, SrvSlot& sl) {
  trioseq_batch_s* bt = sl.batch.get();
  const char* h = reinterpret_cast<const char*>(sl.out.p);
  trioseq_status st = sl.launch_st;
  // A launch that failed part-way may have left work on the stream: drain it before the
  // slot's workspace is reused.
  if (st != TRIOSEQ_OK) cudaStreamSynchronize(sl.stream);
  if (st == TRIOSEQ_OK && cudaEventQuery(sl.done) != cudaSuccess) st = TRIOSEQ_ECUDA;
  int32_t herr = 0;
  if (st == TRIOSEQ_OK) {
    std::memcpy(&herr, h + sl.off_err, 4);
    if (herr & 1) st = TRIOSEQ_ETIMEOUT;
    else if (herr & 2) st = TRIOSEQ_ECUDA;
  }
  const char* alpha = st == TRIOSEQ_OK ? bt->plan->alphabet : nullptr;
  for (size_t i = 0; i < sl.reqs.size(); i++) {
    SrvRes r;
    r.st = st;
    if (st == TRIOSEQ_OK) {
      std::memcpy(&r.score, h + 4 * i, 4);
      const int32_t q = bt->tb_of[i];
      if (q >= 0) {
        int32_t L = 0;
        std::memcpy(&L, h + sl.off_lens + 4 * (size_t)q, 4);
        const int32_t rc = bt->row_cap[q];
        const uint8_t* base =
            reinterpret_cast<const uint8_t*>(h + sl.off_rows + (size_t)bt->row_off[q]);
        r.has_rows = true;
        r.st = no_throw([&] {
          for (int s = 0; s < 3; s++) {
            r.rows[s].resize((size_t)L);
            const uint8_t* row = base + (size_t)s * rc + (rc - L);
            for (int32_t t = 0; t < L; t++) r.rows[s][t] = row[t] == 255 ? '-' : alpha[row[t]];
          }
          return TRIOSEQ_OK;
        });
        if (r.st != TRIOSEQ_OK) {
          r.has_rows = false;
          for (auto& x : r.rows) std::string().swap(x);
        }
      }
    }
    S->done[sl.reqs[i].ticket] = std::move(r);
  }
  sl.reqs.clear();
  sl.batch.reset();
  sl.busy = false;
  S->in_flight -= std::min(S->in_flight, sl.bytes);
  sl.bytes = 0;
}

void srv_loop(trioseq_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool busy_any = false, acted = false;
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      if (sl.launch_st != TRIOSEQ_OK || cudaEventQuery(sl.done) != cudaErrorNotReady) {
        srv_harvest(S, sl);
        acted = true;
      } else {
        busy_any = true;
      }
    }
    for (auto& sl : S->slots) {
      if (sl.busy || S->pending.empty()) continue;
      // Room for a launch on this slot: the budget minus the launches in flight, and with no
      // budget given, no more than the device has free now (plus what this slot already holds,
      // which the launch reuses).
      size_t room = S->budget > S->in_flight ? S->budget - S->in_flight : 0;
      if (S->budget_from_free) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
          room = std::min(room, fr / 10 * 9 + workspace_device_bytes(sl.ws));
        else
          cudaGetLastError();
      }
      bool others_busy = false;
      for (auto& o : S->slots) others_busy = others_busy || o.busy;
      const SrvReq& head = S->pending.front();
      if (head.bytes_alone > room) {
        if (others_busy) break;  // wait: harvested launches give their room back
        if (head.bytes_alone > S->budget) {  // can never fit: fail it alone
          SrvRes r;
          r.st = TRIOSEQ_ENOMEM;
          S->done[head.ticket] = std::move(r);
          S->pending.pop_front();
          acted = true;
          continue;
        }
        // nothing else runs: launch it; its allocations report a real shortage (ENOMEM)
      }
      // Form a launch: the oldest request fixes the group; same-group requests follow in arrival
      // order while the launch's estimate stays within its share of the room.
      const int32_t pid = head.plan_id;
      const uint32_t mode = head.mode;
      const size_t limit = std::max(head.bytes_alone, std::min(room, S->launch_share));
      size_t full = 0;
      std::deque<SrvReq> rest;
      while (!S->pending.empty()) {
        SrvReq& r = S->pending.front();
        const bool same = r.plan_id == pid && r.mode == mode;
        if (sl.reqs.empty() ||
            (same && sl.reqs.size() < S->max_batch && full + r.bytes <= limit)) {
          full += r.bytes;
          sl.reqs.push_back(std::move(r));
        } else {
          rest.push_back(std::move(r));
        }
        S->pending.pop_front();
        if (sl.reqs.size() >= S->max_batch || full >= limit) break;
      }
      while (!rest.empty()) {  // keep arrival order of what was skipped
        S->pending.push_front(std::move(rest.back()));
        rest.pop_back();
      }
      sl.bytes = sl.reqs.size() == 1 ? sl.reqs.front().bytes_alone : full;
      S->in_flight += sl.bytes;
      sl.busy = true;
      acted = true;
      lk.unlock();
      sl.launch_st = no_throw([&] { return srv_launch(S, sl); });  // the thread must not throw
      lk.lock();
      busy_any = true;
    }
    if (S->stop && S->pending.empty() && !busy_any) break;
    if (!acted) S->cv.wait_for(lk, std::chrono::microseconds(busy_any ? 20 : 2000));
  }
}

}  // namespace

extern "C" {

trioseq_status trioseq_server_create(const trioseq_plan_t* plans, int32_t nplans,
                                     size_t hbm_budget, trioseq_server_t* out) {
  return no_throw([&]() -> trioseq_status {
    if (!out) return TRIOSEQ_EINVAL;
    *out = nullptr;
    if (!plans || nplans < 1) return TRIOSEQ_EINVAL;
    for (int32_t i = 0; i < nplans; i++)
      if (!plans[i] || plans[i]->device != plans[0]->device) return TRIOSEQ_EINVAL;
    std::unique_ptr<trioseq_server_s> S(new (std::nothrow) trioseq_server_s());
    if (!S) return TRIOSEQ_ENOMEM;
    S->plans.assign(plans, plans + nplans);
    S->device = plans[0]->device;
    DeviceGuard g(S->device);
    if (hbm_budget == 0) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cuda_status(cudaGetLastError());
      hbm_budget = fr / 10 * 8;
      S->budget_from_free = true;
    }
    S->budget = std::max<size_t>(hbm_budget, 1 << 20);
    S->launch_share = std::max<size_t>(S->budget / trioseq_server_s::kSlots, 1 << 20);
    S->max_pending = (size_t)std::max(0, env_int("TRIOSEQ_SERVER_MAX_PENDING", 1 << 20));
    for (auto& sl : S->slots) {
      if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
        return cuda_status(cudaGetLastError());
      sl.ws.alloc_stream = sl.stream;
    }
    try {
      S->th = std::thread(srv_loop, S.get());
    } catch (...) {
      return TRIOSEQ_ENOMEM;
    }
    *out = S.release();
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_submit(trioseq_server_t S, const trioseq_triplet* t, int32_t plan_id,
                              uint32_t mode, uint64_t* ticket) {
  return no_throw([&]() -> trioseq_status {
    if (!S || !t || !ticket || plan_id < 0 || plan_id >= (int32_t)S->plans.size() ||
        mode > TRIOSEQ_WITH_TRACEBACK)
      return TRIOSEQ_EINVAL;
    const trioseq_plan_s* plan = S->plans[plan_id];
    SrvReq r;
    r.plan_id = plan_id;
    r.mode = mode;
    int64_t sumlen = 0;
    for (int q = 0; q < 3; q++) {
      if (t->len[q] && !t->s[q]) return TRIOSEQ_EINVAL;
      if (t->len[q] > (1u << 24)) return TRIOSEQ_EOVERFLOW;
      const unsigned char* src = reinterpret_cast<const unsigned char*>(t->s[q]);
      for (uint32_t e = 0; e < t->len[q]; e++)
        if (plan->lut[src[e]] < 0) return TRIOSEQ_EINVAL;
      r.s[q].assign(t->s[q] ? t->s[q] : "", t->len[q]);
      sumlen += t->len[q];
    }
    if ((int64_t)std::max(plan->max_abs_sig2, plan->atype != kGlobal ? -2 * plan->gap : 0) *
            sumlen >= (1LL << 26) - 1)
      return TRIOSEQ_EOVERFLOW;
    r.bytes = request_bytes(plan, mode, t->len);
    r.bytes_alone = request_bytes_alone(plan, mode, t->len);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->stop) return TRIOSEQ_EINVAL;
      if (S->pending.size() >= S->max_pending) return TRIOSEQ_EAGAIN;
      r.ticket = S->next_ticket++;
      *ticket = r.ticket;
      S->live[r.ticket] = 0;
      S->pending.push_back(std::move(r));
    }
    S->cv.notify_one();
    return TRIOSEQ_OK;
  });
}

trioseq_status trioseq_poll(trioseq_server_t S, uint64_t ticket, int32_t* score, char* rows[3],
                            size_t cap, size_t* aln_len) {
  return no_throw([&]() -> trioseq_status {
    if (!S) return TRIOSEQ_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) return S->live.count(ticket) ? TRIOSEQ_EAGAIN : TRIOSEQ_EINVAL;
    SrvRes& r = it->second;
    if (r.st == TRIOSEQ_OK && r.has_rows) {
      if (aln_len) *aln_len = r.rows[0].size();
      if (rows) {
        if (cap < r.rows[0].size() || !rows[0] || !rows[1] || !rows[2]) return TRIOSEQ_EINVAL;
        for (int s = 0; s < 3; s++) std::memcpy(rows[s], r.rows[s].data(), r.rows[s].size());
      }
    } else if (aln_len) {
      *aln_len = 0;
    }
    if (score) *score = r.score;
    const trioseq_status st = r.st;
    S->done.erase(it);
    S->live.erase(ticket);
    return st;
  });
}

trioseq_status trioseq_server_destroy(trioseq_server_t S) {
  return no_throw([&]() -> trioseq_status {
    if (!S) return TRIOSEQ_OK;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    {
      DeviceGuard g(S->device);
      for (auto& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        sl.batch.reset();
        sl.ws.release();  // freed in the slot stream's order, while the stream exists
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
      }
    }
    delete S;
    return TRIOSEQ_OK;
  });
}

}  // extern "C"

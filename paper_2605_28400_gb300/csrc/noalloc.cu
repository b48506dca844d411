// noalloc.cu — allocation-free scoring of one triplet (trioseq_align_noalloc).
//
// For callers that must not allocate device memory at call time: processes whose device memory
// is fully reserved up front by another allocator (a framework's caching pool, a fixed budget of
// a serving process), or plugin hosts that forbid cudaMalloc/cudaFree inside their callbacks.
// The call's workspace lives in one file-scope __device__ array of kScratchBytes, which every
// GPU that loads this library holds until the process exits. The caller passes the sequences
// and the score slot in its own device memory; everything else (encoded residues, triplet
// descriptor, work queue, progress flags, boundary records) is placed in that array.
//
// Every call uses the same array and it keeps the last call's contents, so calls that overlap
// on the GPU race: callers must serialise them (one stream, or their own lock plus stream
// order). The flags, queue head and error word are cleared by the set-up kernel of each call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "engine.h"
#include "trioseq.h"

namespace trioseq {
namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kNoallocNJ = 8, kNoallocNK = 8;       // the score-only 8x8 wavefront variant
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NoallocTables {
  int32_t sig[(kMaxAlphabet + 1) * (kMaxAlphabet + 1)];  // sigma'' with the virtual row/column
  int8_t lut[256];                                       // byte -> residue code, -1 invalid
};

struct NoallocLayout {
  size_t off_seq, off_sig, off_desc, off_tasks, off_prog, off_faces, total;
  int nJ, nK, T, ntasks;
};

__host__ __device__ inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Workspace layout of one call, sized in 64-bit arithmetic: the task count nJ * nK of a long,
// thin triplet can exceed 2^31 even though each length is at most 2^24. Returns false when the
// task count or any size does not fit (the caller then reports TRIOSEQ_ESCRATCH); the layout's
// int fields are set only when it fits.
bool layout_for(int64_t a, int64_t b, int64_t c, int KP, NoallocLayout* out) {
  NoallocLayout L{};
  const int64_t WJ = kPR * kNoallocNJ, WK = kPC * kNoallocNK;
  const int64_t nJ = (b + 1 + WJ - 1) / WJ, nK = (c + 1 + WK - 1) / WK;
  const int64_t ntasks = nJ * nK;  // < 2^38 for lengths <= 2^24: no 64-bit overflow
  // Every task holds (a + 1) slices of records, at least one int32 each: a task count beyond
  // the array's int32 capacity can never fit, and rejecting it first keeps the products below
  // (ntasks * (a + 1) * record width) far from 64-bit overflow.
  if (ntasks > (int64_t)(kScratchBytes / sizeof(int32_t))) return false;
  size_t off = 0;
  L.off_seq = off;
  off = up(off + up((size_t)a, 16) + up((size_t)b, 16) + up((size_t)c, 16) + 16, 256);
  L.off_sig = off;
  off = up(off + sizeof(int32_t) * (size_t)KP * KP, 256);
  L.off_desc = off;
  off = up(off + sizeof(TripDesc), 256);
  L.off_tasks = off;
  off = up(off + sizeof(Task) * (size_t)ntasks, 256);
  L.off_prog = off;
  off = up(off + sizeof(int32_t) * ((size_t)ntasks + 64), 256);
  L.off_faces = off;
  off += sizeof(int32_t) * (size_t)ntasks * (size_t)(a + 1) * (size_t)((WK + 4) + WJ);
  L.total = up(off, 256);
  if (L.total > kScratchBytes) return false;
  L.nJ = (int)nJ;
  L.nK = (int)nK;
  L.T = (int)(a + 1 + (kPR - 1) + (kPC - 1));
  L.ntasks = (int)ntasks;
  *out = L;
  return true;
}

// Set-up of one call (after the progress flags, queue head and error word were cleared on the
// same stream): encode the three sequences into the scratch (an invalid byte sets error bit 2
// and encodes as the virtual residue, so the sweep stays in bounds), copy the sigma'' table,
// and write the triplet descriptor and the anti-diagonal-ordered task list.
__global__ void noalloc_setup_kernel(unsigned char* scratch, NoallocLayout L, NoallocTables tab,
                                     int KP, const unsigned char* s0, int a,
                                     const unsigned char* s1, int b, const unsigned char* s2,
                                     int c, int32_t score_base) {
  int8_t* seq = reinterpret_cast<int8_t*>(scratch + L.off_seq);
  int32_t* sig = reinterpret_cast<int32_t*>(scratch + L.off_sig);
  int32_t* prog = reinterpret_cast<int32_t*>(scratch + L.off_prog);
  Task* tasks = reinterpret_cast<Task*>(scratch + L.off_tasks);
  const int o1 = (int)up((size_t)a, 16), o2 = o1 + (int)up((size_t)b, 16);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  int bad = 0;
  for (int e = tid; e < a + b + c; e += nth) {
    const unsigned char ch = e < a ? s0[e] : (e < a + b ? s1[e - a] : s2[e - a - b]);
    int code = tab.lut[ch];
    if (code < 0) {
      bad = 1;
      code = KP - 1;
    }
    const int dst = e < a ? e : (e < a + b ? o1 + (e - a) : o2 + (e - a - b));
    seq[dst] = (int8_t)code;
  }
  for (int e = tid; e < KP * KP; e += nth) sig[e] = tab.sig[e];
  // task q of the queue: anti-diagonal D = J + K ascending, J ascending within D
  for (int q = tid; q < L.ntasks; q += nth) {
    const int J = q / L.nK, K = q % L.nK, D = J + K;
    int rank = 0;
    for (int d = 0; d < D; ++d) {  // tasks on earlier anti-diagonals
      const int lo = max(0, d - (L.nK - 1)), hi = min(L.nJ - 1, d);
      rank += hi >= lo ? hi - lo + 1 : 0;
    }
    rank += J - max(0, D - (L.nK - 1));
    tasks[rank] = Task{0, J, K, 0};
  }
  if (tid == 0) {
    TripDesc d{};
    d.s_off[0] = 0;
    d.s_off[1] = o1;
    d.s_off[2] = o2;
    d.oj_off = 0;
    d.ok_off = (int64_t)L.ntasks * (a + 1) * (kPC * kNoallocNK + 4);
    d.code_off = -1;
    d.prog_base = 0;
    d.len[0] = a;
    d.len[1] = b;
    d.len[2] = c;
    d.glen[0] = a;
    d.glen[1] = b;
    d.glen[2] = c;
    d.pair = -1;
    d.nJ = L.nJ;
    d.nK = L.nK;
    d.T = L.T;
    d.score_base = score_base;
    d.out_idx = 0;
    d.tb_idx = -1;
    *reinterpret_cast<TripDesc*>(scratch + L.off_desc) = d;
  }
  if (bad) atomicOr(prog + L.ntasks + 32, 4);
}

std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

}  // namespace
}  // namespace trioseq

using namespace trioseq;

extern "C" trioseq_status trioseq_align_noalloc(const trioseq_scoring* sc,
                                                const unsigned char* d_s0, uint32_t a,
                                                const unsigned char* d_s1, uint32_t b,
                                                const unsigned char* d_s2, uint32_t c,
                                                int32_t* d_score, void* stream) {
  if (!sc || !sc->alphabet || !sc->sub || !d_score) return TRIOSEQ_EINVAL;
  if ((a && !d_s0) || (b && !d_s1) || (c && !d_s2)) return TRIOSEQ_EINVAL;
  const int K = sc->alphabet_size;
  if (K < 1 || K > kMaxAlphabet || sc->gap > 0 || sc->gap < -127) return TRIOSEQ_EINVAL;
  const int KP = K + 1;
  NoallocTables tab;
  for (int i = 0; i < 256; i++) tab.lut[i] = -1;
  for (int i = 0; i < KP * KP; i++) tab.sig[i] = 0;
  int32_t mx = 1;
  for (int i = 0; i < K; i++) {
    const unsigned char ch = (unsigned char)sc->alphabet[i];
    if (tab.lut[ch] >= 0) return TRIOSEQ_EINVAL;
    tab.lut[ch] = (int8_t)i;
    for (int j = 0; j < K; j++) {
      if (sc->sub[i * K + j] != sc->sub[j * K + i]) return TRIOSEQ_EINVAL;
      const int32_t v = (int32_t)sc->sub[i * K + j] - 2 * sc->gap;
      tab.sig[i * KP + j] = v;
      mx = v > mx ? v : (-v > mx ? -v : mx);
    }
  }
  const int64_t sumlen = (int64_t)a + b + c;
  if (a > (1u << 24) || b > (1u << 24) || c > (1u << 24)) return TRIOSEQ_ESCRATCH;
  if ((int64_t)mx * sumlen >= (1LL << 26) - 1) return TRIOSEQ_EOVERFLOW;
  NoallocLayout L{};
  if (!layout_for(a, b, c, KP, &L)) return TRIOSEQ_ESCRATCH;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TRIOSEQ_ECUDA;
  }
  unsigned char* scratch = nullptr;
  {
    // Set-up once per device, with that device current: the host-side name of the array is a
    // stand-in, so the kernels get the device address looked up here.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return TRIOSEQ_ECUDA;
      }
      g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t score_base = 2 * sc->gap * (int32_t)sumlen;
  if (cudaMemsetAsync(scratch + L.off_prog, 0, sizeof(int32_t) * ((size_t)L.ntasks + 64), st) !=
      cudaSuccess) {
    cudaGetLastError();
    return TRIOSEQ_ECUDA;
  }
  noalloc_setup_kernel<<<64, 256, 0, st>>>(scratch, L, tab, KP, d_s0, (int)a, d_s1, (int)b, d_s2,
                                           (int)c, score_base);
  if (cudaGetLastError() != cudaSuccess) return TRIOSEQ_ECUDA;

  int sms = 0, bpm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return TRIOSEQ_ECUDA;
  }
  const size_t smem = wavefront_smem_bytes(kNoallocNJ, kNoallocNK, KP, false);
  if (wavefront_occupancy(kNoallocNJ, kNoallocNK, false, kGlobal, false, false, smem, &bpm) != 0 ||
      bpm <= 0)
    return TRIOSEQ_ECUDA;
  int32_t* prog = reinterpret_cast<int32_t*>(scratch + L.off_prog);
  WaveParams p{};
  p.desc = reinterpret_cast<const TripDesc*>(scratch + L.off_desc);
  p.tasks = reinterpret_cast<const Task*>(scratch + L.off_tasks);
  p.ntasks = L.ntasks;
  p.KP = KP;
  p.seq = reinterpret_cast<const int8_t*>(scratch + L.off_seq);
  p.sig = reinterpret_cast<const int32_t*>(scratch + L.off_sig);
  p.faces = reinterpret_cast<int32_t*>(scratch + L.off_faces);
  p.progress = prog;
  p.queue = prog + L.ntasks;
  p.codes = nullptr;
  p.scores = d_score;
  p.err = prog + L.ntasks + 32;
  p.TI = 8;
  p.g2 = -2 * sc->gap;
  p.one = 1;
  p.wait_ns = 2000000000LL;
  if (launch_wavefront(kNoallocNJ, kNoallocNK, false, kGlobal, false, false, p, sms * bpm, smem,
                       st) != 0) {
    cudaGetLastError();
    return TRIOSEQ_ECUDA;
  }
  int32_t herr = 0;
  if (cudaMemcpyAsync(&herr, p.err, sizeof(herr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return TRIOSEQ_ECUDA;
  }
  if (herr & 4) return TRIOSEQ_EINVAL;
  if (herr & 1) return TRIOSEQ_ETIMEOUT;
  return TRIOSEQ_OK;
}

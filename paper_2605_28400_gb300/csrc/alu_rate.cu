// alu_rate.cu — measured issue rate of the int32 instruction forms the cell update is built from.
//
// The wavefront kernel's roofline counts 13 int32 operations per cell (7 adds, 6 maxima) against
// SMs x 128 int32 lanes x SM clock. This file measures what the GPU actually sustains for each
// form the kernel issues: a plain maximum, the fused add-maximum (__viaddmax_s32, max(a + b, c)),
// the 3-input maximum (__vimax3_s32), a 3-input add, and a multiply-add by a runtime 1 (how the
// kernel moves adds to the FMA pipe). One wave of blocks fills every SM to its occupancy limit
// and each thread runs 8 interleaved recurrences, so the measurement sees throughput, not
// latency. Each block records its SM and its start and end clock; an SM's rate is its blocks'
// instructions over its busy span (first start to last end: co-resident blocks finish at very
// different times under the warp scheduler). CUDA events give the wall time, hence the clock.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "trioseq.h"
#include "guard.h"

using trioseq::no_throw;

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int OP>
__device__ __forceinline__ int step(int x, int y, int z, int b, int one) {
  if constexpr (OP == 0) return max(x, y);
  if constexpr (OP == 1) return __viaddmax_s32(y, b, x);  // max(y + b, x)
  if constexpr (OP == 2) return __vimax3_s32(x, y, z);
  if constexpr (OP == 3) return x + y + b;
  int d;
  asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(y), "r"(one), "r"(x));
  return d;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) alu_rate_kernel(int iters, int b, int one, int* sink,
                                                             long long* stamps) {
  int acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = (int)(threadIdx.x * 7 + k * 13 + blockIdx.x);
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    // chain k reads its neighbours' previous values: kChains independent updates per round
    int nxt[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      nxt[k] = step<OP>(acc[k], acc[(k + 1) % kChains], acc[(k + 2) % kChains], b, one);
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = nxt[k];
  }
  __syncthreads();
  const long long t1 = clock64();
  int s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= acc[k];
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
  if (threadIdx.x == 0) {  // SM id, start and end clock of this block
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    stamps[3 * blockIdx.x] = (long long)smid;
    stamps[3 * blockIdx.x + 1] = t0;
    stamps[3 * blockIdx.x + 2] = t1;
  }
}

template <int OP>
cudaError_t launch(int grid, int iters, int* sink, long long* stamps, cudaStream_t st) {
  alu_rate_kernel<OP><<<grid, kThreads, 0, st>>>(iters, -1, 1, sink, stamps);
  return cudaGetLastError();
}

template <int OP>
int occupancy() {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, alu_rate_kernel<OP>, kThreads, 0) !=
      cudaSuccess)
    return 0;
  return blocks;
}

}  // namespace

extern "C" trioseq_status trioseq_alu_rate(int32_t op, double* per_clk_per_sm, double* sm_mhz) {
  return no_throw([&]() -> trioseq_status {
    if (op < 0 || op > 4 || !per_clk_per_sm || !sm_mhz) return TRIOSEQ_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return TRIOSEQ_ECUDA;
    }
    // one wave: every SM holds its resident maximum of blocks for the whole run
    const int per_sm = op == 0   ? occupancy<0>()
                       : op == 1 ? occupancy<1>()
                       : op == 2 ? occupancy<2>()
                       : op == 3 ? occupancy<3>()
                                 : occupancy<4>();
    if (per_sm <= 0) {
      cudaGetLastError();
      return TRIOSEQ_ECUDA;
    }
    const int grid = sms * per_sm;
    const int iters = 1 << 14;
    int* sink = nullptr;
    long long* stamps = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    trioseq_status status = TRIOSEQ_ECUDA;
    std::vector<long long> stm(3 * (size_t)grid);
    float ms = 0.f;
    const auto run = [&](cudaStream_t s) -> cudaError_t {
      switch (op) {
        case 0: return launch<0>(grid, iters, sink, stamps, s);
        case 1: return launch<1>(grid, iters, sink, stamps, s);
        case 2: return launch<2>(grid, iters, sink, stamps, s);
        case 3: return launch<3>(grid, iters, sink, stamps, s);
        default: return launch<4>(grid, iters, sink, stamps, s);
      }
    };
    do {
      if (cudaMalloc(&sink, sizeof(int) * (size_t)grid * kThreads) != cudaSuccess ||
          cudaMalloc(&stamps, sizeof(long long) * 3 * (size_t)grid) != cudaSuccess ||
          cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        break;
      if (run(st) != cudaSuccess) break;  // warm-up (clocks up, code loaded)
      if (cudaEventRecord(e0, st) != cudaSuccess || run(st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          cudaMemcpy(stm.data(), stamps, sizeof(long long) * 3 * (size_t)grid,
                     cudaMemcpyDeviceToHost) != cudaSuccess)
        break;
      // per SM: blocks it ran, first start, last end (its own clock)
      std::vector<long long> first(1024, -1), last(1024, -1), nblk(1024, 0);
      bool bad = false;
      for (int g = 0; g < grid && !bad; g++) {
        const long long sm = stm[3 * (size_t)g], t0 = stm[3 * (size_t)g + 1],
                        t1 = stm[3 * (size_t)g + 2];
        if (sm < 0 || sm >= 1024) {
          bad = true;
          break;
        }
        first[sm] = first[sm] < 0 ? t0 : std::min(first[sm], t0);
        last[sm] = std::max(last[sm], t1);
        nblk[sm]++;
      }
      if (bad) break;
      std::vector<double> rates, spans;
      for (int sm = 0; sm < 1024; sm++)
        if (nblk[sm] > 0 && last[sm] > first[sm]) {
          const double span = (double)(last[sm] - first[sm]);
          rates.push_back((double)nblk[sm] * kThreads * (double)iters * kChains / span);
          spans.push_back(span);
        }
      if (rates.empty()) break;
      std::sort(rates.begin(), rates.end());
      *per_clk_per_sm = rates[rates.size() / 2];  // median over SMs
      const double max_span = *std::max_element(spans.begin(), spans.end());
      *sm_mhz = ms > 0 ? max_span / ((double)ms * 1e3) : 0.0;
      status = TRIOSEQ_OK;
    } while (false);
    if (status != TRIOSEQ_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (stamps) cudaFree(stamps);
    if (sink) cudaFree(sink);
    return status;
  });
}

// Work partitioning of a triplet set over ranks (one rank per GPU), host code only.
//
// Sec. V-D distributes independent triplets over GPUs in three ways:
//  - blocked: the set in dataset order is cut into one contiguous chunk per rank;
//  - interleaved: triplet t goes to rank t mod N (round robin);
//  - dynamic: triplets are taken in dataset order and each goes to the rank whose cumulative
//    cell count is the least so far (the amount of computation is the paper's cell count,
//    |S0|*|S1|*|S2|, Sec. V-A). Ties go to the lowest rank.
// The paper gives no chunk rule for blocked: chunk r here is [floor(r*n/N), floor((r+1)*n/N)),
// so chunk sizes differ by at most one. A fourth scheme, largest first, applies the dynamic rule
// to the triplets in order of decreasing cell count (ties in dataset order): Graham's LPT list
// scheduling, whose largest load is at most 4/3 - 1/(3N) times the optimum; in dataset order a
// few large triplets arriving last can leave one rank far above the rest.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <utility>
#include <vector>

#include "trioseq.h"
#include "guard.h"

using trioseq::no_throw;

// far above any GPU count; keeps the per-rank arrays small
constexpr int32_t kMaxRanks = 1 << 20;

extern "C" trioseq_status trioseq_partition(const uint32_t* lens, size_t n, int32_t nranks,
                                            int32_t scheme, int32_t* rank_of,
                                            uint64_t* cells_per_rank) {
  return no_throw([&]() -> trioseq_status {
    if (nranks < 1 || nranks > kMaxRanks || (n && (!lens || !rank_of))) return TRIOSEQ_EINVAL;
    if (scheme != TRIOSEQ_PART_BLOCKED && scheme != TRIOSEQ_PART_INTERLEAVED &&
        scheme != TRIOSEQ_PART_DYNAMIC && scheme != TRIOSEQ_PART_LARGEST_FIRST)
      return TRIOSEQ_EINVAL;
    // the whole set's cell count must fit 64 bits, so every rank's load does too
    unsigned __int128 total = 0;
    for (size_t t = 0; t < n; t++)
      total += (unsigned __int128)lens[3 * t] * lens[3 * t + 1] * lens[3 * t + 2];
    if (total > (unsigned __int128)UINT64_MAX) return TRIOSEQ_EOVERFLOW;
    const uint64_t N = (uint64_t)nranks;
    std::vector<uint64_t> load(N, 0);
    auto cells = [&](size_t t) {
      return (uint64_t)lens[3 * t] * lens[3 * t + 1] * lens[3 * t + 2];
    };
    if (scheme == TRIOSEQ_PART_BLOCKED) {
      // rank r owns [floor(r n / N), floor((r+1) n / N)); walk the boundaries once
      uint64_t r = 0;
      for (size_t t = 0; t < n; t++) {
        while ((unsigned __int128)(r + 1) * n / N <= t) r++;
        rank_of[t] = (int32_t)r;
        load[r] += cells(t);
      }
    } else if (scheme == TRIOSEQ_PART_INTERLEAVED) {
      for (size_t t = 0; t < n; t++) {
        rank_of[t] = (int32_t)(t % N);
        load[t % N] += cells(t);
      }
    } else {
      // the order triplets are taken in: dataset order, or decreasing cells (stable)
      std::vector<size_t> order(n);
      for (size_t t = 0; t < n; t++) order[t] = t;
      if (scheme == TRIOSEQ_PART_LARGEST_FIRST)
        std::stable_sort(order.begin(), order.end(),
                         [&](size_t x, size_t y) { return cells(x) > cells(y); });
      // least cumulative cells first, then the lowest rank: a min-heap on (load, rank)
      using Entry = std::pair<uint64_t, int32_t>;
      std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
      for (int32_t r = 0; r < nranks; r++) heap.push({0, r});
      for (size_t t : order) {
        Entry e = heap.top();
        heap.pop();
        rank_of[t] = e.second;
        e.first += cells(t);
        load[e.second] = e.first;
        heap.push(e);
      }
    }
    if (cells_per_rank)
      for (uint64_t r = 0; r < N; r++) cells_per_rank[r] = load[r];
    return TRIOSEQ_OK;
  });
}

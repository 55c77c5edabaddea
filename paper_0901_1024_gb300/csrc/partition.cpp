// Element numbering for flux-gather locality: the greedy breadth-first
// partition of Section 5.2 ("Flux Extraction"), Algorithm 2.  Blocks of at
// most `block` elements are grown one at a time: the candidate queue starts
// at a seed, each step takes the queued element sharing the most faces with
// the block (ties: the one queued first), and the face neighbours of every
// element taken join the queue (at most once at a time).  A full block hands
// the head of its queue on as the next seed; a dry queue takes the
// lowest-numbered element not yet placed, as does the very first block.
#include <cstdint>
#include <vector>

#include "dg_internal.h"

namespace dg {

void greedy_partition_order(const std::vector<int32_t>& nbr, int64_t K, int64_t block,
                            int64_t* perm) {
  std::vector<uint8_t> placed(K, 0), queued(K, 0);
  std::vector<int32_t> shared(K, 0);        // faces shared with the current block
  std::vector<int64_t> touched;             // entries of `shared` to reset
  std::vector<int64_t> queue;
  int64_t lowest = 0, n_placed = 0, carry = -1;
  auto next_unplaced = [&]() {
    while (lowest < K && placed[lowest]) ++lowest;
    return lowest;
  };
  auto enqueue = [&](int64_t e) {
    if (!queued[e]) {
      queued[e] = 1;
      queue.push_back(e);
    }
  };
  while (n_placed < K) {
    const int64_t seed = carry >= 0 ? carry : next_unplaced();
    carry = -1;
    for (int64_t e : queue) queued[e] = 0;
    queue.clear();
    for (int64_t e : touched) shared[e] = 0;
    touched.clear();
    enqueue(seed);
    int64_t filled = 0;
    for (;;) {
      size_t best = 0;
      for (size_t i = 1; i < queue.size(); ++i)
        if (shared[queue[i]] > shared[queue[best]]) best = i;
      const int64_t e = queue[best];
      queue.erase(queue.begin() + static_cast<std::ptrdiff_t>(best));
      queued[e] = 0;
      if (!placed[e]) {
        placed[e] = 1;
        perm[n_placed++] = e;
        ++filled;
        for (int f = 0; f < 4; ++f) {
          const int64_t n = nbr[4 * e + f];
          if (n >= 0 && n != e) {
            if (shared[n]++ == 0) touched.push_back(n);
          }
        }
        if (filled == block) {
          if (!queue.empty()) carry = queue.front();
          break;
        }
        for (int f = 0; f < 4; ++f) {
          const int64_t n = nbr[4 * e + f];
          if (n >= 0 && n != e) enqueue(n);
        }
      }
      if (queue.empty()) {
        if (n_placed == K) break;
        enqueue(next_unplaced());
      }
    }
  }
}

}  // namespace dg

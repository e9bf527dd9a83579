// Work-unit scheduler of the serving runtime (host code only; tested on the CPU through
// tests/sched_driver.cpp).  The paper has no counterpart: its energies are distributed over
// ranks once per iteration (Sec. 4.4).
//
// A request is split into work units, one per energy chunk; the units of a request are
// independent solves (different energies of the same device).  The scheduler picks the next
// unit to start when a worker is free:
//   * round robin over the requests that still have units to start: the request whose unit was
//     started least recently (in arrival order at first) goes first, so every admitted request
//     progresses chunk by chunk and a large request does not hold the device until it ends;
//   * a request whose unit does not fit in the arena's free memory now is skipped and the next
//     one is tried (small units pass a blocked one);
//   * no starvation: the first request in round-robin order (the head) counts the units started
//     past it while it did not fit; once that count reaches max_skips nothing else is started
//     until the head fits.
#pragma once
#include <cstddef>
#include <vector>

namespace bt {

struct SchedEntry {
  long long order = 0;   // round-robin key: smaller goes first (arrival order, then restart order)
  int units_left = 0;    // units not yet started
  size_t bytes = 0;      // workspace of one unit
  int skips = 0;         // units started past this entry while it was the head and did not fit
};

// Index of the entry whose next unit starts now, or -1 (nothing can start).  `fits(bytes)` asks
// the arena whether a block of that size can be allocated now.  On success the caller starts the
// unit, decrements units_left and gives the entry a new order key after every other entry's.
template <class Fits>
int sched_pick(std::vector<SchedEntry>& entries, int max_skips, Fits fits) {
  int head = -1;
  for (int i = 0; i < (int)entries.size(); ++i)
    if (entries[i].units_left > 0 && (head < 0 || entries[i].order < entries[head].order)) head = i;
  if (head < 0) return -1;
  if (fits(entries[head].bytes)) {
    entries[head].skips = 0;
    return head;
  }
  if (entries[head].skips >= max_skips) return -1;  // the head waits for memory; nothing passes it
  // the others in round-robin order
  int best = -1;
  for (int i = 0; i < (int)entries.size(); ++i) {
    if (i == head || entries[i].units_left <= 0 || !fits(entries[i].bytes)) continue;
    if (best < 0 || entries[i].order < entries[best].order) best = i;
  }
  if (best >= 0) ++entries[head].skips;
  return best;
}

}  // namespace bt

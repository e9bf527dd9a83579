// Test driver of the serving scheduler (csrc/unit_sched.h), host code only.
// stdin:  "E n max_skips" then n lines "order units bytes"; then commands
//         "P free"   pick with `free` bytes available (fits(b) == b <= free); prints the index or
//                    -1; a pick decrements the entry's units and moves it behind every other entry
//         "A units bytes"   add an entry (a request arriving later: behind every other entry)
// stdout: one integer per P command.
#include <iostream>
#include <string>
#include <vector>

#include "unit_sched.h"

int main() {
  std::string cmd;
  int n = 0, max_skips = 0;
  std::cin >> cmd >> n >> max_skips;
  std::vector<bt::SchedEntry> e(n);
  long long seq = 1000000;
  for (auto& x : e) std::cin >> x.order >> x.units_left >> x.bytes;
  while (std::cin >> cmd) {
    if (cmd == "P") {
      size_t free_bytes = 0;
      std::cin >> free_bytes;
      const int i = bt::sched_pick(e, max_skips, [&](size_t b) { return b <= free_bytes; });
      if (i >= 0) {
        --e[i].units_left;
        e[i].order = ++seq;
      }
      std::cout << i << "\n";
    } else if (cmd == "A") {
      bt::SchedEntry x;
      std::cin >> x.units_left >> x.bytes;
      x.order = ++seq;
      e.push_back(x);
    }
  }
  return 0;
}

// Host-only driver for the serving arena (csrc/arena.h), built with g++ by test_arena_cpu.py.
// Reads commands from stdin, one per line:
//   reset <bytes>       start over with an empty arena of <bytes>
//   alloc <bytes>       prints the offset, or -1 when nothing fits
//   release <off> <bytes>
#include <cstdio>
#include <cstring>

#include "arena.h"

int main() {
  bt::Arena a;
  char cmd[32];
  while (std::scanf("%31s", cmd) == 1) {
    if (!std::strcmp(cmd, "reset")) {
      unsigned long long n;
      if (std::scanf("%llu", &n) != 1) return 2;
      a.reset(nullptr, (size_t)n);
    } else if (!std::strcmp(cmd, "alloc")) {
      unsigned long long n;
      if (std::scanf("%llu", &n) != 1) return 2;
      const size_t off = a.alloc((size_t)n);
      if (off == SIZE_MAX)
        std::printf("-1\n");
      else
        std::printf("%llu\n", (unsigned long long)off);
    } else if (!std::strcmp(cmd, "release")) {
      unsigned long long off, n;
      if (std::scanf("%llu %llu", &off, &n) != 2) return 2;
      a.release((size_t)off, (size_t)n);
    } else {
      return 3;
    }
  }
  return 0;
}

// First-fit arena over one device allocation, used by the serving loop (server.cu) to lend each
// admitted request its workspace out of the memory budget reserved at create.  Host code only:
// it hands out offsets and never touches the memory.  Blocks are rounded up to 256 bytes; the
// free list (offset -> length) is kept coalesced, so the free space is always exactly the gaps
// between live blocks and an arena whose blocks are all released is one free range again.
#pragma once
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>

namespace bt {

class Arena {
 public:
  void reset(char* base, size_t bytes) {
    base_ = base;
    free_.clear();
    free_[0] = bytes;
  }
  // returns offset or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  // whether alloc(bytes) would succeed now
  bool can_alloc(size_t bytes) const {
    bytes = (bytes + 255) / 256 * 256;
    for (const auto& kv : free_)
      if (kv.second >= bytes) return true;
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* base() const { return base_; }

 private:
  char* base_ = nullptr;
  std::map<size_t, size_t> free_;  // offset -> length
};

}  // namespace bt

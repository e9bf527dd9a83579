// Measurement aid, not part of the solver: a launch list of the device work of a region of a
// program from CUPTI's activity records (device start / end timestamps of every kernel, memcpy
// and memset, graph-launched kernels included), collected in process, without a profiler that
// serialises or replays launches.  Built on demand (kernel_driver --kernel steptrace) into its
// own shared library linked against libcupti; the solver library does not depend on it.
//
//   bt_trace_start()   registers the buffer callbacks and enables the activity kinds
//   bt_trace_stop()    flushes every buffer and disables them
//   bt_trace_count() / bt_trace_get(i, ...)   the records collected, in completion order
#include <cupti.h>
#include <cxxabi.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace {

struct Rec {
  std::string name;
  unsigned long long start, end;
  int kind;  // 0 kernel, 1 memcpy, 2 memset
};

std::string demangle(const char* n) {
  if (!n) return "?";
  int st = 0;
  char* d = abi::__cxa_demangle(n, nullptr, nullptr, &st);
  std::string out = (st == 0 && d) ? std::string(d) : std::string(n);
  free(d);
  return out;
}

std::mutex g_mu;
std::vector<Rec> g_recs;
constexpr size_t kBufBytes = 8u << 20;

void CUPTIAPI buffer_requested(uint8_t** buffer, size_t* size, size_t* max_records) {
  void* p = nullptr;
  if (posix_memalign(&p, 8, kBufBytes) != 0) p = nullptr;
  *buffer = static_cast<uint8_t*>(p);
  *size = p ? kBufBytes : 0;
  *max_records = 0;
}

void CUPTIAPI buffer_completed(CUcontext, uint32_t, uint8_t* buffer, size_t, size_t valid) {
  CUpti_Activity* rec = nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  while (buffer && cuptiActivityGetNextRecord(buffer, valid, &rec) == CUPTI_SUCCESS) {
    if (rec->kind == CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL || rec->kind == CUPTI_ACTIVITY_KIND_KERNEL) {
      const auto* k = reinterpret_cast<const CUpti_ActivityKernel10*>(rec);
      g_recs.push_back(Rec{demangle(k->name), (unsigned long long)k->start, (unsigned long long)k->end, 0});
    } else if (rec->kind == CUPTI_ACTIVITY_KIND_MEMCPY) {
      const auto* m = reinterpret_cast<const CUpti_ActivityMemcpy6*>(rec);
      g_recs.push_back(Rec{"memcpy", (unsigned long long)m->start, (unsigned long long)m->end, 1});
    } else if (rec->kind == CUPTI_ACTIVITY_KIND_MEMSET) {
      const auto* m = reinterpret_cast<const CUpti_ActivityMemset4*>(rec);
      g_recs.push_back(Rec{"memset", (unsigned long long)m->start, (unsigned long long)m->end, 2});
    }
  }
  free(buffer);
}

}  // namespace

extern "C" int bt_trace_start(void) {
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_recs.clear();
  }
  if (cuptiActivityRegisterCallbacks(buffer_requested, buffer_completed) != CUPTI_SUCCESS) return 1;
  if (cuptiActivityEnable(CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL) != CUPTI_SUCCESS) return 2;
  if (cuptiActivityEnable(CUPTI_ACTIVITY_KIND_MEMCPY) != CUPTI_SUCCESS) return 3;
  if (cuptiActivityEnable(CUPTI_ACTIVITY_KIND_MEMSET) != CUPTI_SUCCESS) return 4;
  return 0;
}

extern "C" int bt_trace_stop(void) {
  if (cuptiActivityFlushAll(1) != CUPTI_SUCCESS) return 1;
  cuptiActivityDisable(CUPTI_ACTIVITY_KIND_CONCURRENT_KERNEL);
  cuptiActivityDisable(CUPTI_ACTIVITY_KIND_MEMCPY);
  cuptiActivityDisable(CUPTI_ACTIVITY_KIND_MEMSET);
  return 0;
}

extern "C" int bt_trace_count(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  return (int)g_recs.size();
}

// Record i: its name (truncated to name_len - 1 characters), device start and end (ns) and kind
// (0 kernel, 1 memcpy, 2 memset); returns -1 when i is out of range.
extern "C" int bt_trace_get(int i, char* name, int name_len, unsigned long long* start, unsigned long long* end) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (i < 0 || i >= (int)g_recs.size()) return -1;
  const Rec& r = g_recs[(size_t)i];
  if (name && name_len > 0) {
    std::strncpy(name, r.name.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = '\0';
  }
  if (start) *start = r.start;
  if (end) *end = r.end;
  return r.kind;
}

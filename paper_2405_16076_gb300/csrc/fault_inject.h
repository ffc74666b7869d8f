// Host-side allocation-failure injection (no device fault is involved): RID_FAULT_INJECT=alloc:<n>
// makes the n-th device allocation after it is armed report out-of-memory, once.  Plain C++ with no
// CUDA dependency, so that the parsing and the countdown are tested on their own.
#pragma once
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

namespace rid {

// n of "alloc:<n>" (n >= 1); 0 (off) for anything else, including NULL.
inline int64_t parse_fault_inject(const char* v) {
  if (!v || strncmp(v, "alloc:", 6) != 0) return 0;
  char* end = nullptr;
  const long long n = strtoll(v + 6, &end, 10);
  if (end == v + 6 || *end != '\0' || n < 1) return 0;
  return (int64_t)n;
}

// Counts allocations down from n; the call that takes it from 1 to 0 is the one that fails.
struct AllocCountdown {
  std::atomic<int64_t> left{0};
  void arm(int64_t n) { left.store(n > 0 ? n : 0); }
  bool next_fails() {
    if (left.load(std::memory_order_relaxed) <= 0) return false;
    return left.fetch_sub(1) == 1;
  }
};

}  // namespace rid

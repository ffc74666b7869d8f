// Host-side failure injection (no device fault is involved): RID_FAULT_INJECT=alloc:<n> makes the
// n-th device allocation after it is armed report out-of-memory, once; RID_FAULT_INJECT=wait:<n>
// shortens the poll limit of the tensor-core pipeline waits of new handles to n.  Plain C++ with no
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

// n of "wait:<n>" (1 <= n <= 2^22): the poll limit of the tensor-core kernels' pipeline waits in
// handles created while it is set, so that a test can make a bounded wait give up (the kernel then
// raises the timeout bit of the device error word, drains and returns); 0 (off) otherwise.
inline uint32_t parse_wait_inject(const char* v) {
  if (!v || strncmp(v, "wait:", 5) != 0) return 0;
  char* end = nullptr;
  const long long n = strtoll(v + 5, &end, 10);
  if (end == v + 5 || *end != '\0' || n < 1 || n > (1LL << 22)) return 0;
  return (uint32_t)n;
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

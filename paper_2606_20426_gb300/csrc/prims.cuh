// Device primitives used at scene setup: scan, stable radix sort,
// compaction, bounding box.  All are deterministic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace tc {

// Device-memory arena of one env: every allocation goes through the
// caller-provided tc_allocator (e.g. a PyTorch caching allocator) or
// cudaMallocAsync on the env's stream.
struct Arena {
  tc_allocator user{};
  bool has_user = false;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  struct Block { void* p; size_t n; };
  std::vector<Block> live;

  void* get(size_t n);
  void put(void* p);
  void release_all();
  template <class T> T* alloc(int64_t count) {
    return static_cast<T*>(get(sizeof(T) * (size_t)(count > 0 ? count : 1)));
  }
};

// out[i] = sum_{j<i} in[j]; returns the total (synchronises the stream).
int64_t scan_exclusive(const int32_t* in, int32_t* out, int64_t n, Arena& a);

// Stable LSD radix sort of (keys, vals) on the low `bits` bits of the keys.
void radix_sort(uint64_t* keys, uint32_t* vals, int64_t n, int bits, Arena& a);

// Bounding box of n double points (SoA) -> host lo[3], hi[3].
void bbox(const double* x, const double* y, const double* z, int64_t n, double lo[3], double hi[3],
          Arena& a);

}  // namespace tc

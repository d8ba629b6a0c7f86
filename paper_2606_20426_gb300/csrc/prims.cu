// Setup-time device primitives: exclusive scan, stable LSD radix sort,
// bounding box, and the env memory arena.
#include <algorithm>

#include "prims.cuh"

namespace tc {

// ------------------------------------------------------------------ arena

void* Arena::get(size_t n) {
  n = (n + 255) & ~size_t(255);
  void* p = nullptr;
  if (has_user) {
    p = user.alloc(user.ctx, n, (void*)stream);
  } else {
    if (cudaMallocAsync(&p, n, stream) != cudaSuccess) p = nullptr;
  }
  if (p) {
    live.push_back({p, n});
    bytes += n;
  }
  return p;
}

void Arena::put(void* p) {
  if (!p) return;
  for (size_t i = 0; i < live.size(); ++i) {
    if (live[i].p == p) {
      if (has_user) user.release(user.ctx, p, live[i].n, (void*)stream);
      else cudaFreeAsync(p, stream);
      bytes -= live[i].n;
      live[i] = live.back();
      live.pop_back();
      return;
    }
  }
}

void Arena::release_all() {
  for (auto& b : live) {
    if (has_user) user.release(user.ctx, b.p, b.n, (void*)stream);
    else cudaFreeAsync(b.p, stream);
  }
  live.clear();
  bytes = 0;
}

// ------------------------------------------------------------------- scan

constexpr int kScanBlock = 512;

__global__ void k_block_sums(const int32_t* in, int64_t n, int64_t* sums) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  double v = i < n ? (double)in[i] : 0.0;
  v = block_sum<kScanBlock>(v);
  if (threadIdx.x == 0) sums[blockIdx.x] = (int64_t)v;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nb, int64_t* total) {
  // one block: sequential chunks with a block-wide prefix per chunk
  __shared__ int64_t s[kScanBlock];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanBlock) {
    const int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? sums[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
      int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + s[threadIdx.x] - v;  // exclusive
    carry += s[kScanBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_blocks(const int32_t* in, int32_t* out, int64_t n, const int64_t* sums) {
  __shared__ int64_t s[kScanBlock];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = (int32_t)(sums[blockIdx.x] + s[threadIdx.x] - v);
}

int64_t scan_exclusive(const int32_t* in, int32_t* out, int64_t n, Arena& a) {
  if (n <= 0) return 0;
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  int64_t* sums = a.alloc<int64_t>(nb + 1);
  k_block_sums<<<(unsigned)nb, kScanBlock, 0, a.stream>>>(in, n, sums);
  k_scan_sums<<<1, kScanBlock, 0, a.stream>>>(sums, nb, sums + nb);
  k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, a.stream>>>(in, out, n, sums);
  int64_t total = 0;
  cudaMemcpyAsync(&total, sums + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, a.stream);
  cudaStreamSynchronize(a.stream);
  a.put(sums);
  return total;
}

// -------------------------------------------------------------- radix sort
//
// One tile of 256 elements per block, 8 warps.  Ranks within a tile come from
// __match_any_sync (peers with the same digit in the warp) and per-warp digit
// counts, so the scatter preserves the input order of equal digits.

constexpr int kRadixBlock = 256;
constexpr int kRadixWarps = kRadixBlock / 32;

struct TileRank {
  int digit;
  int local;  // rank among equal digits inside the tile
};

__device__ TileRank tile_rank(uint32_t digit, bool valid, int (*cnt)[256], int* tile_total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadixWarps * 256; d += kRadixBlock) (&cnt[0][0])[d] = 0;
  __syncthreads();
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 0xffffffffu) & act;
  int rank_w = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank_w == 0) cnt[w][digit] = __popc(peers);
  __syncthreads();
  // prefix over warps for each digit (thread d handles digit d)
  {
    const int d = threadIdx.x;  // kRadixBlock == 256 digits
    int run = 0;
    for (int k = 0; k < kRadixWarps; ++k) {
      const int c = cnt[k][d];
      cnt[k][d] = run;
      run += c;
    }
    tile_total[d] = run;
  }
  __syncthreads();
  TileRank r;
  r.digit = (int)digit;
  r.local = valid ? cnt[w][digit] + rank_w : 0;
  return r;
}

__global__ void k_radix_hist(const uint64_t* keys, int64_t n, int shift, int32_t* hist, int64_t ntiles) {
  __shared__ int cnt[kRadixWarps][256];
  __shared__ int tot[256];
  const int64_t i = (int64_t)blockIdx.x * kRadixBlock + threadIdx.x;
  const bool valid = i < n;
  const uint32_t dg = valid ? (uint32_t)((keys[i] >> shift) & 0xffu) : 0u;
  tile_rank(dg, valid, cnt, tot);
  // digit-major layout: hist[d * ntiles + tile]
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = tot[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* keys, const uint32_t* vals, int64_t n, int shift,
                                const int32_t* offs, int64_t ntiles, uint64_t* okeys, uint32_t* ovals) {
  __shared__ int cnt[kRadixWarps][256];
  __shared__ int tot[256];
  const int64_t i = (int64_t)blockIdx.x * kRadixBlock + threadIdx.x;
  const bool valid = i < n;
  uint64_t k = valid ? keys[i] : 0;
  const uint32_t dg = valid ? (uint32_t)((k >> shift) & 0xffu) : 0u;
  TileRank r = tile_rank(dg, valid, cnt, tot);
  if (valid) {
    const int64_t pos = (int64_t)offs[(int64_t)dg * ntiles + blockIdx.x] + r.local;
    okeys[pos] = k;
    ovals[pos] = vals[i];
  }
}

void radix_sort(uint64_t* keys, uint32_t* vals, int64_t n, int bits, Arena& a) {
  if (n <= 1) return;
  const int64_t ntiles = (n + kRadixBlock - 1) / kRadixBlock;
  int32_t* hist = a.alloc<int32_t>(256 * ntiles);
  int32_t* offs = a.alloc<int32_t>(256 * ntiles);
  uint64_t* k2 = a.alloc<uint64_t>(n);
  uint32_t* v2 = a.alloc<uint32_t>(n);
  uint64_t *ki = keys, *ko = k2;
  uint32_t *vi = vals, *vo = v2;
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_radix_hist<<<(unsigned)ntiles, kRadixBlock, 0, a.stream>>>(ki, n, shift, hist, ntiles);
    scan_exclusive(hist, offs, 256 * ntiles, a);
    k_radix_scatter<<<(unsigned)ntiles, kRadixBlock, 0, a.stream>>>(ki, vi, n, shift, offs, ntiles, ko, vo);
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  if (ki != keys) {
    cudaMemcpyAsync(keys, ki, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, a.stream);
    cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, a.stream);
  }
  cudaStreamSynchronize(a.stream);
  a.put(hist);
  a.put(offs);
  a.put(k2);
  a.put(v2);
}

// -------------------------------------------------------------------- bbox

__global__ void k_bbox(const double* x, const double* y, const double* z, int64_t n, double* out) {
  const double* c[3] = {x, y, z};
  for (int d = 0; d < 3; ++d) {
    double lo = 1e308, hi = -1e308;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      lo = fmin(lo, c[d][i]);
      hi = fmax(hi, c[d][i]);
    }
    lo = block_min<kBlock>(lo);
    hi = block_max<kBlock>(hi);
    if (threadIdx.x == 0) {
      out[(blockIdx.x * 3 + d) * 2 + 0] = lo;
      out[(blockIdx.x * 3 + d) * 2 + 1] = hi;
    }
  }
}

void bbox(const double* x, const double* y, const double* z, int64_t n, double lo[3], double hi[3], Arena& a) {
  const int nb = 64;
  double* part = a.alloc<double>(nb * 6);
  k_bbox<<<nb, kBlock, 0, a.stream>>>(x, y, z, n, part);
  std::vector<double> h(nb * 6);
  cudaMemcpyAsync(h.data(), part, sizeof(double) * nb * 6, cudaMemcpyDeviceToHost, a.stream);
  cudaStreamSynchronize(a.stream);
  a.put(part);
  for (int d = 0; d < 3; ++d) {
    lo[d] = 1e308;
    hi[d] = -1e308;
    for (int b = 0; b < nb; ++b) {
      lo[d] = std::min(lo[d], h[(b * 3 + d) * 2 + 0]);
      hi[d] = std::max(hi[d], h[(b * 3 + d) * 2 + 1]);
    }
  }
}

}  // namespace tc

// Deterministic exclusive prefix sum (int32 or int64 input, int64 output) in three
// passes: tile sums, a single-block scan of the tile sums, and the in-tile scan.
#include "internal.h"

namespace ephb {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

__device__ inline int64_t block_exclusive(int64_t v, int64_t *sh, int64_t &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < (kScanThreads / 32) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kScanThreads / 32)) sh[lane] = w;
  }
  __syncthreads();
  int64_t before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
  total = sh[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const T *in, int64_t n, int64_t *bsum) {
  __shared__ int64_t sh[32];
  int64_t base = int64_t(blockIdx.x) * kTile + int64_t(threadIdx.x) * kScanItems;
  int64_t s = 0;
  for (int j = 0; j < kScanItems; ++j)
    if (base + j < n) s += int64_t(in[base + j]);
  int64_t total;
  block_exclusive(s, sh, total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t *bsum, int64_t nb, int64_t *total_out) {
  __shared__ int64_t sh[32];
  int64_t carry = 0;
  for (int64_t c = 0; c < nb; c += kScanThreads) {
    int64_t i = c + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive(v, sh, tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T *in, int64_t n, const int64_t *boff,
                                                            int64_t *out) {
  __shared__ int64_t sh[32];
  int64_t base = int64_t(blockIdx.x) * kTile + int64_t(threadIdx.x) * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? int64_t(in[base + j]) : 0;
    s += v[j];
  }
  int64_t total;
  int64_t ex = block_exclusive(s, sh, total) + boff[blockIdx.x];
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = ex;
    ex += v[j];
  }
}

}  // namespace

int64_t scan_scratch_elems(int64_t n) { return (n + kTile - 1) / kTile + 1; }

template <typename T>
cudaError_t exclusive_scan(const T *in, int64_t *out, int64_t n, int64_t *total_dev, int64_t *scratch,
                           int64_t scratch_elems, cudaStream_t st) {
  if (n <= 0) {
    if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(int64_t), st);
    return cudaSuccess;
  }
  int64_t nb = (n + kTile - 1) / kTile;
  if (nb > scratch_elems) return cudaErrorInvalidValue;
  EPHB_LAUNCH(k_tile_sums<T>, unsigned(nb), kScanThreads, 0, st, in, n, scratch);
  EPHB_LAUNCH(k_scan_sums, 1, kScanThreads, 0, st, scratch, nb, total_dev);
  EPHB_LAUNCH(k_tile_scan<T>, unsigned(nb), kScanThreads, 0, st, in, n, scratch, out);
  return cudaGetLastError();
}

template cudaError_t exclusive_scan<int>(const int *, int64_t *, int64_t, int64_t *, int64_t *, int64_t,
                                         cudaStream_t);
template cudaError_t exclusive_scan<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *, int64_t *, int64_t,
                                             cudaStream_t);

}  // namespace ephb

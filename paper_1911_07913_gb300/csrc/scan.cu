// Device-wide exclusive prefix sums (reduce -> scan of block sums -> scan),
// used for counting-sort offsets and stream compaction.
#include "internal.h"

namespace hot {

namespace {
constexpr int SCAN_NT = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_ITEMS;

template <class In>
__global__ void k_tile_sums(const In *__restrict__ in, int64_t n, int *__restrict__ sums) {
  __shared__ int sh[SCAN_NT / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int acc = 0;
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_NT) {
    int64_t i = base + k;
    if (i < n) acc += (int)in[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < SCAN_NT / 32; ++w) t += sh[w];
    sums[blockIdx.x] = t;
  }
}

// one block: exclusive scan of nb tile sums in place, total in *total
__global__ void k_scan_sums(int *__restrict__ sums, int nb, int *__restrict__ total) {
  __shared__ int sh[1024 / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int w = sh[threadIdx.x];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (threadIdx.x >= o) w += y;
      }
      sh[threadIdx.x] = w;
    }
    __syncthreads();
    int warp_prefix = (threadIdx.x >> 5) ? sh[(threadIdx.x >> 5) - 1] : 0;
    int c = carry;
    if (i < nb) sums[i] = c + warp_prefix + x - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + warp_prefix + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class In>
__global__ void k_tile_scan(const In *in, int64_t n, const int *__restrict__ sums, int *out) {
  __shared__ int sh[SCAN_NT / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int tsum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? (int)in[i] : 0;
    tsum += v[k];
  }
  int x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  if ((threadIdx.x & 31) == 31) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = threadIdx.x < SCAN_NT / 32 ? sh[threadIdx.x] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (threadIdx.x >= o) w += y;
    }
    if (threadIdx.x < SCAN_NT / 32) sh[threadIdx.x] = w;
  }
  __syncthreads();
  int run = sums[blockIdx.x] + ((threadIdx.x >> 5) ? sh[(threadIdx.x >> 5) - 1] : 0) + x - tsum;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

template <class In>
void scan_impl(const In *in, int *out, int64_t n, ScanScratch &sc, cudaStream_t st) {
  sc.total.ensure(1);
  if (n <= 0) {
    HOT_CUDA(cudaMemsetAsync(sc.total.p, 0, sizeof(int), st));
    return;
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  sc.block_sums.ensure(nb);
  k_tile_sums<In><<<(unsigned)nb, SCAN_NT, 0, st>>>(in, n, sc.block_sums.p);
  HOT_LAUNCH("k_tile_sums");
  k_scan_sums<<<1, 1024, 0, st>>>(sc.block_sums.p, (int)nb, sc.total.p);
  HOT_LAUNCH("k_scan_sums");
  k_tile_scan<In><<<(unsigned)nb, SCAN_NT, 0, st>>>(in, n, sc.block_sums.p, out);
  HOT_LAUNCH("k_tile_scan");
}
}  // namespace

void exclusive_scan(const int *in, int *out, int64_t n, ScanScratch &sc, cudaStream_t st) {
  scan_impl<int>(in, out, n, sc, st);
}
void exclusive_scan_u8(const uint8_t *in, int *out, int64_t n, ScanScratch &sc, cudaStream_t st) {
  scan_impl<uint8_t>(in, out, n, sc, st);
}
int read_scan_total(ScanScratch &sc, cudaStream_t st) {
  int t = 0;
  HOT_CUDA(cudaMemcpyAsync(&t, sc.total.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  HOT_CUDA(cudaStreamSynchronize(st));
  return t;
}

}  // namespace hot

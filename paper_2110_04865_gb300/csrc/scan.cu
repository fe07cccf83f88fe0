// Device-wide exclusive prefix sums of int64 arrays whose length lives in
// device memory (so the same launches can sit inside a captured CUDA graph
// while the length changes from round to round).
//
// Reduce-then-scan over a fixed grid of NB_SCAN blocks: block b owns the
// contiguous chunk [b*C, (b+1)*C) with C = ceil(N / NB_SCAN); pass 1 sums each
// chunk, pass 2 scans the NB_SCAN chunk sums in one block, pass 3 rescans each
// chunk from its offset.  Traffic: 2 reads + 1 write per element.
#include "internal.cuh"

namespace msf {

namespace {

constexpr int SCAN_THREADS = 256;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// Inclusive scan across the block; returns the thread's inclusive value and
// the block total in *total.
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_sums[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int64_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
    s = warp_incl_scan(s);
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  if (wid > 0) v += warp_sums[wid - 1];
  *total = warp_sums[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return v;
}

__device__ __forceinline__ void chunk_of(int64_t N, int64_t *lo, int64_t *hi) {
  const int64_t C = (N + NB_SCAN - 1) / NB_SCAN;
  *lo = (int64_t)blockIdx.x * C;
  *hi = *lo + C < N ? *lo + C : N;
  if (*lo > N) *lo = N;
}

// Array pointers are given directly or, when the *_ind argument is not NULL,
// read from device memory (the compaction scans run inside a CUDA graph that
// serves many problems, so their arrays are only known on the device).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int64_t *in, int64_t *const *in_ind,
                                                                const int64_t *n_dev, int64_t *tmp,
                                                                int64_t *const *tmp_ind) {
  if (in_ind) in = *in_ind;
  if (tmp_ind) tmp = *tmp_ind;
  int64_t lo, hi;
  chunk_of(*n_dev, &lo, &hi);
  int64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += SCAN_THREADS) s += in[i];
  int64_t tot;
  block_incl_scan(s, &tot);
  if (threadIdx.x == 0) tmp[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(NB_SCAN) k_scan_top(int64_t *tmp, int64_t *const *tmp_ind, int64_t *total_dev) {
  if (tmp_ind) tmp = *tmp_ind;
  __shared__ int64_t warp_sums[NB_SCAN / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t v = tmp[threadIdx.x];
  int64_t x = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = warp_sums[lane];
    s = warp_incl_scan(s);
    warp_sums[lane] = s;
  }
  __syncthreads();
  if (wid > 0) x += warp_sums[wid - 1];
  tmp[threadIdx.x] = x - v;  // exclusive
  if (threadIdx.x == NB_SCAN - 1) {
    tmp[NB_SCAN] = x;
    if (total_dev) *total_dev = x;
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const int64_t *in, int64_t *const *in_ind,
                                                              int64_t *out, int64_t *const *out_ind,
                                                              const int64_t *n_dev, const int64_t *tmp,
                                                              int64_t *const *tmp_ind) {
  if (in_ind) in = *in_ind;
  if (out_ind) out = *out_ind;
  if (tmp_ind) tmp = *tmp_ind;
  int64_t lo, hi;
  chunk_of(*n_dev, &lo, &hi);
  int64_t carry = tmp[blockIdx.x];
  for (int64_t base = lo; base < hi; base += SCAN_THREADS) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < hi ? in[i] : 0;
    int64_t tot;
    const int64_t incl = block_incl_scan(v, &tot);
    if (i < hi) out[i] = carry + incl - v;
    carry += tot;
  }
}

}  // namespace

void launch_scan_excl(const int64_t *in, int64_t *out, const int64_t *n_dev, int64_t *tmp,
                      int64_t *total_dev, cudaStream_t s) {
  k_scan_reduce<<<NB_SCAN, SCAN_THREADS, 0, s>>>(in, nullptr, n_dev, tmp, nullptr);
  k_scan_top<<<1, NB_SCAN, 0, s>>>(tmp, nullptr, total_dev);
  k_scan_down<<<NB_SCAN, SCAN_THREADS, 0, s>>>(in, nullptr, out, nullptr, n_dev, tmp, nullptr);
}

void launch_scan_excl_ind(int64_t *const *inout_ind, const int64_t *n_dev, int64_t *const *tmp_ind,
                          int64_t *total_dev, cudaStream_t s) {
  k_scan_reduce<<<NB_SCAN, SCAN_THREADS, 0, s>>>(nullptr, inout_ind, n_dev, nullptr, tmp_ind);
  k_scan_top<<<1, NB_SCAN, 0, s>>>(nullptr, tmp_ind, total_dev);
  k_scan_down<<<NB_SCAN, SCAN_THREADS, 0, s>>>(nullptr, inout_ind, nullptr, inout_ind, n_dev, nullptr, tmp_ind);
}

}  // namespace msf

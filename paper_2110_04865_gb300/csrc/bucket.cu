// Bucketed CSR builder.
//
// Same result as the per-vertex atomic builder (both directions of every
// non-loop edge grouped by row; slot order inside a row arbitrary), built so
// that the per-vertex counters live in shared memory and the global writes
// are coalesced or confined to a small window of the slot arrays:
//
//   1. every block validates its contiguous chunk of edges (endpoint
//      table) and counts the records (one per direction) of each bucket of
//      2^S consecutive rows;
//   2. an exclusive scan of the (bucket, block) counts gives every block a
//      private range per bucket; the block sorts tiles of its records by
//      bucket in shared memory and writes each bucket's run contiguously, so
//      bucket b's records (row, col, key) end up in the slot range that
//      bucket b's rows occupy in the CSR;
//   3. work items (runs of one bucket's records) count their rows in shared
//      memory and add the counts to the vertex degrees (one global atomic per
//      distinct row and item);
//   4. rows[] and rp[] from the degrees (rows_from_degrees);
//   5. the same work items count again, claim one run of slots per distinct
//      row from the row's cursor (one global atomic per distinct row and
//      item) and place their records.  Items are taken in bucket order, so
//      the slots being written at any time form a window of the slot arrays
//      that stays in L2 while its sectors fill up.
//
// Random 4- and 8-byte writes spread over a slot array much larger than L2
// are slow on GB300 (each partial sector is read back from DRAM), and so are
// same-address global atomics on high-degree vertices; both are avoided.
#include "internal.cuh"

namespace msf {

namespace {

constexpr int BT = 256;          // threads per block (passes 1, 3, 5)
constexpr int BTV = 1024;        // threads per block of the validation (pass 1)
constexpr int BT1 = 512;         // threads per block of the bucket scatter (pass 2)
constexpr int BT2 = 512;         // threads per block of the sub-bucket scatter
constexpr int TE = 4608;         // edges per tile of the bucket scatter
constexpr int EPT = TE / BT1;    // edges per thread and tile
constexpr int VMAX = 4096;       // vertices per bucket at most (2^S)
constexpr int NBMAX = 1024;      // buckets at most
constexpr int ITEM3 = 16384;     // records per work item of pass 3
constexpr int ITEM5 = 4096;      // records per work item of pass 5 over sub-buckets (512 rows)
constexpr int BT5 = 512;         // threads per block of pass 5 over sub-buckets
constexpr int ITEM5N = 8192;     // the same over buckets of 2048 or 4096 rows: larger items meet
constexpr int BT5N = 1024;       // more records per row, so fewer rows claim a run per record
constexpr uint32_t NOREC = 0xffffffffu;

// Records between the bucket scatter and the item passes: (row, column) as
// two words, or packed into one word, column << S | bucket-local row, when
// the column needs at most 32 - S bits (PACK).  The key travels beside it.
template <bool PACK>
__device__ __forceinline__ void rec_store(void *rc, uint64_t pos, uint32_t row, uint32_t col, int S) {
  if (PACK) reinterpret_cast<uint32_t *>(rc)[pos] = (col << S) | (row & ((1u << S) - 1u));
  else reinterpret_cast<uint2 *>(rc)[pos] = make_uint2(row, col);
}
// (row, column) of record i; with PACK the row is bucket-local
template <bool PACK>
__device__ __forceinline__ uint2 rec_load(const void *rc, int64_t i, int S) {
  if (PACK) {
    const uint32_t w = __ldcs(reinterpret_cast<const uint32_t *>(rc) + i);
    return make_uint2(w & ((1u << S) - 1u), w >> S);
  }
  return __ldcs(reinterpret_cast<const uint2 *>(rc) + i);
}
// row of record i (bucket-local with PACK)
template <bool PACK>
__device__ __forceinline__ uint32_t rec_row(const void *rc, int64_t i, int S) {
  if (PACK) return __ldcs(reinterpret_cast<const uint32_t *>(rc) + i) & ((1u << S) - 1u);
  return __ldcs(&reinterpret_cast<const uint2 *>(rc)[i].x);
}

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Asks L2 for the bytes of elements [lo, hi) of a device array of
// `elem`-byte elements (one bulk prefetch, a hint with no effect on
// results), rounded out to 16-byte boundaries but kept below byte
// elem * lim, the end of the array's data.  Only for the library's own
// buffers (device memory); does nothing unless `a` is 16-byte aligned.
__device__ __forceinline__ void l2_prefetch(const void *a, int elem, int64_t lo, int64_t hi, int64_t lim) {
  if (reinterpret_cast<uintptr_t>(a) & 15u) return;
  const uint64_t b0 = ((uint64_t)lo * elem) & ~15ull;
  uint64_t b1 = ((uint64_t)hi * elem + 15u) & ~15ull;
  const uint64_t end = ((uint64_t)lim * elem) & ~15ull;
  if (b1 > end) b1 = end;
  if (lo < 0 || b1 <= b0) return;
  uint64_t n = b1 - b0;
  if (n > (1u << 30)) n = 1u << 30;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char *>(a) + b0),
               "r"((uint32_t)n)
               : "memory");
}

// edges [lo, hi) of the block for passes 1 and 2
__device__ __forceinline__ void edge_chunk(int64_t m, int64_t E, int64_t *lo, int64_t *hi) {
  *lo = (int64_t)blockIdx.x * E;
  *hi = min64(*lo + E, m);
  if (*hi < *lo) *hi = *lo;
}

// Pass 1 fused with the validation of the endpoints: block k validates its
// chunk of edges [k*E, (k+1)*E) (endpoint table, count of non-loop edges)
// and counts the records of each bucket.  The weights are checked for NaN
// by the bucket scatter, which reads them anyway (a NaN edge keeps its
// records; the build then fails).  VEC: src, dst 16-byte aligned and E a
// multiple of 4 -- four edges per thread and step with 16-byte loads and
// stores.  Block 0 also stores the histogram's length for the scan (*hlen).
template <bool VEC>
__global__ void __launch_bounds__(BTV) k_bk_validate(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                                    int wtype, int64_t m, int64_t n,
                                                    int32_t G, const int64_t *eoff, const int64_t *voff, int64_t E,
                                                    int nb, int S, int2 *__restrict__ ends, int *err,
                                                    unsigned long long *nonloop, long long *H,
                                                    long long *hlen) {
  __shared__ unsigned hist[NBMAX];
  if (blockIdx.x == 0 && threadIdx.x == 0) *hlen = (long long)nb * gridDim.x;
  for (int i = threadIdx.x; i < nb; i += BTV) hist[i] = 0;
  __syncthreads();
  int64_t lo, hi;
  edge_chunk(m, E, &lo, &hi);
  unsigned cnt = 0;
  auto one = [&](int64_t e, int32_t u, int32_t v) -> int2 {
    const int2 uv = validate_edge(e, u, v, 0u, wtype, n, G, eoff, voff, err);
    if (uv.x != uv.y) {
      ++cnt;
      atomicAdd(hist + (uv.x >> S), 1u);
      atomicAdd(hist + (uv.y >> S), 1u);
    }
    return uv;
  };
  int64_t e0 = lo;
  if (VEC) {
    // two quads of edges per thread and step, both loaded first (64 bytes in
    // flight per thread: with one quad the pass streamed at 5 TB/s, what
    // 32 bytes per thread of 32 warps per SM sustain at DRAM latency)
    const int64_t q1 = hi >> 2;
    const int4 *s4p = reinterpret_cast<const int4 *>(src), *d4p = reinterpret_cast<const int4 *>(dst);
    auto quad = [&](int64_t q, int4 s4, int4 d4) {
      const int64_t e = q << 2;
      const int2 a = one(e, s4.x, d4.x);
      const int2 b = one(e + 1, s4.y, d4.y);
      const int2 c = one(e + 2, s4.z, d4.z);
      const int2 d = one(e + 3, s4.w, d4.w);
      int4 *o = reinterpret_cast<int4 *>(ends + e);
      o[0] = make_int4(a.x, a.y, b.x, b.y);
      o[1] = make_int4(c.x, c.y, d.x, d.y);
    };
    for (int64_t q = (lo >> 2) + threadIdx.x; q < q1; q += 2 * BTV) {
      const bool two = q + BTV < q1;
      const int4 s4 = __ldcs(s4p + q), d4 = __ldcs(d4p + q);
      int4 s5 = make_int4(0, 0, 0, 0), d5 = make_int4(0, 0, 0, 0);
      if (two) {
        s5 = __ldcs(s4p + q + BTV);
        d5 = __ldcs(d4p + q + BTV);
      }
      quad(q, s4, d4);
      if (two) quad(q + BTV, s5, d5);
    }
    e0 = q1 << 2 > lo ? q1 << 2 : lo;
  }
  for (int64_t e = e0 + threadIdx.x; e < hi; e += BTV) ends[e] = one(e, src[e], dst[e]);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nonloop, (unsigned long long)cnt);
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += BTV) H[(int64_t)i * gridDim.x + blockIdx.x] = hist[i];
}

// Exclusive scan, in place, of a[0..len) (len a multiple of NT) by a block
// of NT threads; thread t owns the entries [t*P, (t+1)*P).  Returns the
// total.  Ends with the block synchronised.
template <int NT>
__device__ unsigned block_scan_excl(unsigned *a, int len) {
  __shared__ unsigned wtot[NT / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int P = len / NT;
  unsigned s = 0;
  for (int k = 0; k < P; ++k) s += a[t * P + k];
  unsigned incl = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned o = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) wtot[wid] = incl;
  __syncthreads();
  unsigned wpre = 0, total = 0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) {
    const unsigned v = wtot[k];
    if (k < wid) wpre += v;
    total += v;
  }
  unsigned run = wpre + incl - s;
  for (int k = 0; k < P; ++k) {
    const unsigned v = a[t * P + k];
    a[t * P + k] = run;
    run += v;
  }
  __syncthreads();
  return total;
}


// Shared memory of the bucket scatter: the tile sorted by bucket (row and
// column, key), then per bucket the running global position (u64), the
// count and the run start (u32 each; nbp = nb rounded up to BT1).
__host__ __device__ constexpr size_t scatter_smem(int nbp) { return (size_t)2 * TE * 16 + (size_t)nbp * 16; }

// Pass 2.  O = exclusive scan of H; block k writes its records of bucket b to
// [O[b * nblk + k], ...), one coalesced run per (tile, bucket): the record
// (rec_store) and key = ord(w) << 32 | e.
template <bool PACK>
__global__ void __launch_bounds__(BT1) k_bk_scatter(const int2 *__restrict__ ends, const uint32_t *__restrict__ w,
                                                   int wtype, int64_t m, int64_t E, int nb, int nbp, int S,
                                                   const long long *__restrict__ O, void *__restrict__ rc,
                                                   uint64_t *__restrict__ rkey, int *err) {
  extern __shared__ __align__(16) unsigned char bk_raw[];
  uint4 *tile = reinterpret_cast<uint4 *>(bk_raw);  // (row, col, key low, key high)
  unsigned long long *gbase = reinterpret_cast<unsigned long long *>(tile + 2 * TE);
  unsigned *cnt = reinterpret_cast<unsigned *>(gbase + nbp);
  unsigned *start = cnt + nbp;
  for (int i = threadIdx.x; i < nbp; i += BT1) {
    gbase[i] = i < nb ? (unsigned long long)O[(int64_t)i * gridDim.x + blockIdx.x] : 0ull;
    cnt[i] = 0;
  }
  __syncthreads();
  int64_t lo, hi;
  edge_chunk(m, E, &lo, &hi);
  // the tile's edges and weights, loaded one tile ahead
  int2 uv[EPT], nuv[EPT];
  uint32_t wv[EPT], nwv[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int64_t e = lo + threadIdx.x + (int64_t)k * BT1;
    nuv[k] = e < hi ? __ldcs(ends + e) : make_int2(0, 0);
    nwv[k] = e < hi ? __ldcs(w + e) : 0u;
  }
  for (int64_t t0 = lo; t0 < hi; t0 += TE) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      uv[k] = nuv[k];
      wv[k] = nwv[k];
      const int64_t e = t0 + TE + threadIdx.x + (int64_t)k * BT1;
      nuv[k] = e < hi ? __ldcs(ends + e) : make_int2(0, 0);
      nwv[k] = e < hi ? __ldcs(w + e) : 0u;
    }
    // the NaN check of the weights (the validation reads only endpoints)
    bool nan = false;
#pragma unroll
    for (int k = 0; k < EPT; ++k) nan |= wtype == MSF_F32 && (wv[k] & 0x7fffffffu) > 0x7f800000u;
    if (nan) atomicOr(err, 2);
    // rank both records of every non-loop edge in its bucket
    unsigned rk[2 * EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if (uv[k].x != uv[k].y) {
        rk[2 * k] = atomicAdd(cnt + (uv[k].x >> S), 1u);
        rk[2 * k + 1] = atomicAdd(cnt + (uv[k].y >> S), 1u);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbp; i += BT1) start[i] = cnt[i];
    __syncthreads();
    const unsigned total = block_scan_excl<BT1>(start, nbp);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if (uv[k].x == uv[k].y) continue;
      const int64_t e = t0 + threadIdx.x + (int64_t)k * BT1;
      const uint32_t kh = ord_weight_dev(wv[k], wtype), kl = (uint32_t)e;
      tile[start[uv[k].x >> S] + rk[2 * k]] = make_uint4((uint32_t)uv[k].x, (uint32_t)uv[k].y, kl, kh);
      tile[start[uv[k].y >> S] + rk[2 * k + 1]] = make_uint4((uint32_t)uv[k].y, (uint32_t)uv[k].x, kl, kh);
    }
    __syncthreads();
    // record i of the sorted tile goes to its bucket's next place
    for (unsigned i = threadIdx.x; i < total; i += BT1) {
      const uint4 x = tile[i];
      const int b = (int)(x.x >> S);
      const unsigned long long pos = gbase[b] + (i - start[b]);
      rec_store<PACK>(rc, pos, x.x, x.y, S);
      rkey[pos] = ((uint64_t)x.w << 32) | x.z;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbp; i += BT1) {
      gbase[i] += cnt[i];
      cnt[i] = 0;
    }
    __syncthreads();
  }
}

// Work items: bucket b's records [bs_b, be_b) are cut into ceil(size / item)
// items; item_start[b] = items of the buckets before b, item_start[nb] =
// total.  One block of 1024 threads; the second item size and list (item2,
// item_start2) are optional.
__device__ void bk_items(const long long *O, int nb, int nblk, const long long *nnz, int item,
                         long long *item_start) {
  __shared__ long long wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long carry = 0;
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int b = b0 + threadIdx.x;
    long long c = 0;
    if (b < nb) {
      const long long bs = O[(int64_t)b * nblk];
      const long long be = (b + 1 < nb) ? O[(int64_t)(b + 1) * nblk] : *nnz;
      c = (be - bs + item - 1) / item;
    }
    long long v = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long o = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += o;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
      long long s = wsum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, s, d);
        if (lane >= d) s += o;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    const long long excl = carry + (wid > 0 ? wsum[wid - 1] : 0) + v - c;
    if (b < nb) item_start[b] = excl;
    carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) item_start[nb] = carry;
}
__global__ void __launch_bounds__(1024) k_bk_items(const long long *O, int nb, int nblk, const long long *nnz,
                                                   int item, long long *item_start, int item2,
                                                   long long *item_start2) {
  bk_items(O, nb, nblk, nnz, item, item_start);
  if (item_start2) {
    __syncthreads();
    bk_items(O, nb, nblk, nnz, item2, item_start2);
  }
}

// The item counts of groups [0, ng) on every SM, for the groups of the
// sub-bucket path (131 072 at 2^26 vertices: one block took 250 us over
// them): c1[g] and c2[g] = the group's records in items of 2^sh1 and 2^sh2,
// which an exclusive scan of each then turns into item starts.  Block 0
// stores ng for the scans.
__global__ void __launch_bounds__(BT) k_bk_counts(const long long *O, int ng, int gstride, const long long *nnz,
                                                  int sh1, long long *c1, int sh2, long long *c2,
                                                  long long *n_dev) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_dev = ng;
  const long long tot = *nnz;
  const int64_t stride = (int64_t)gridDim.x * BT;
  for (int64_t b = (int64_t)blockIdx.x * BT + threadIdx.x; b < ng; b += stride) {
    const long long bs = O[b * gstride];
    const long long be = (b + 1 < ng) ? O[(b + 1) * gstride] : tot;
    const long long len = be - bs;
    c1[b] = (len + (1ll << sh1) - 1) >> sh1;
    c2[b] = (len + (1ll << sh2) - 1) >> sh2;
  }
}

// imap[it] = the bucket of item `it` (k_bk_item_map): one load instead of a
// binary search over item_start, whose dependent steps stalled every item.
// One warp per bucket (a hub bucket has thousands of items); the second
// list and map (item_start2, imap2) are optional.
__global__ void __launch_bounds__(BT) k_bk_item_map(const long long *item_start, int nb, int *imap,
                                                    const long long *item_start2, int *imap2) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (BT / 32);
  for (int64_t b = (int64_t)blockIdx.x * (BT / 32) + (threadIdx.x >> 5); b < nb; b += warps) {
    const long long i1 = item_start[b + 1];
    for (long long it = item_start[b] + lane; it < i1; it += 32) imap[it] = (int)b;
    if (imap2) {
      const long long j1 = item_start2[b + 1];
      for (long long it = item_start2[b] + lane; it < j1; it += 32) imap2[it] = (int)b;
    }
  }
}

// Item `it`: its bucket, record range [lo, hi) and the bucket's first record.
__device__ __forceinline__ int item_range(const long long *item_start, const int *imap, int nb, const long long *O,
                                          int nblk, const long long *nnz, int item, long long it, int64_t *lo,
                                          int64_t *hi, int64_t *bs) {
  const int l = imap[it];
  const int64_t s0 = O[(int64_t)l * nblk];
  const int64_t s1 = (l + 1 < nb) ? O[(int64_t)(l + 1) * nblk] : *nnz;
  *bs = s0;
  *lo = s0 + (it - item_start[l]) * item;
  *hi = min64(*lo + item, s1);
  return l;
}

// Pass 3.  deg[v] += records of row v in the item (the owner of each
// counter adds it once and clears it).
template <bool PACK>
__global__ void __launch_bounds__(BT) k_bk_degree(const long long *item_start, const int *imap, int nb,
                                                  const long long *O,
                                                  int nblk, const long long *nnz, const void *__restrict__ rc,
                                                  int S, int64_t n, unsigned *deg) {
  __shared__ unsigned cnt[VMAX];
  const int V = 1 << S, P = V / BT;
  for (int i = threadIdx.x; i < V; i += BT) cnt[i] = 0;
  __syncthreads();
  const long long T = item_start[nb];
  const uint32_t lmask = (uint32_t)V - 1u;
  for (long long it = blockIdx.x; it < T; it += gridDim.x) {
    int64_t lo, hi, bs;
    const int b = item_range(item_start, imap, nb, O, nblk, nnz, ITEM3, it, &lo, &hi, &bs);
    // 16-byte words of RPW records; the ragged ends (fewer than RPW records
    // each) record by record
    constexpr int RPW = PACK ? 4 : 2;
    const int64_t w0 = (lo + RPW - 1) / RPW, w1 = hi / RPW;  // whole words [w0, w1)
    if (w0 >= w1) {
      for (int64_t i = lo + threadIdx.x; i < hi; i += BT) atomicAdd(cnt + (rec_row<PACK>(rc, i, S) & lmask), 1u);
    } else {
      const int64_t h1 = w0 * RPW, t0 = w1 * RPW;
      if (threadIdx.x < h1 - lo) atomicAdd(cnt + (rec_row<PACK>(rc, lo + threadIdx.x, S) & lmask), 1u);
      if (threadIdx.x < hi - t0) atomicAdd(cnt + (rec_row<PACK>(rc, t0 + threadIdx.x, S) & lmask), 1u);
      const uint4 *wp = reinterpret_cast<const uint4 *>(rc);
      for (int64_t q0 = w0 + threadIdx.x; q0 < w1; q0 += 4 * BT) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t q = q0 + (int64_t)k * BT;
          v[k] = q < w1 ? __ldcs(wp + q) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (q0 + (int64_t)k * BT >= w1) continue;
          atomicAdd(cnt + (v[k].x & lmask), 1u);  // the row: the low S bits (PACK) or the first word
          atomicAdd(cnt + (v[k].z & lmask), 1u);
          if (PACK) {
            atomicAdd(cnt + (v[k].y & lmask), 1u);
            atomicAdd(cnt + (v[k].w & lmask), 1u);
          }
        }
      }
    }
    __syncthreads();
    const int64_t v0 = (int64_t)b << S;
    for (int k = 0; k < P; ++k) {
      const int j = threadIdx.x * P + k;
      const unsigned c = cnt[j];
      if (c) {
        if (v0 + j < n) atomicAdd(deg + v0 + j, c);
        cnt[j] = 0;
      }
    }
    __syncthreads();
  }
}

// Shared memory of the placement: per bucket-local row the count (then the
// row's start in the sorted item) and the row's run offset inside the
// bucket's slot range; the item sorted by row (local row, column, key).
__host__ __device__ constexpr size_t place_smem(int V, int item) { return (size_t)V * 8 + (size_t)item * 14; }

// Pass 5.  cursor[v] = next free slot of row v (rp at the start).  The item
// is sorted by row in shared memory; each distinct row claims one run of
// slots from its cursor; the sorted records are written run by run.
template <int P, bool PACK, int NT, int ITEM>  // rows per counter owner: 2^S = P * NT
__global__ void __launch_bounds__(NT, 1024 / NT) k_bk_place(const long long *item_start, const int *imap, int nb,
                                                     const long long *O,
                                                 int nblk, const long long *nnz, const void *__restrict__ rc,
                                                 const uint64_t *__restrict__ rkey, int S, int64_t n,
                                                 unsigned long long *cursor, int32_t *__restrict__ col,
                                                 uint64_t *__restrict__ key) {
  extern __shared__ __align__(16) unsigned char bk_raw[];
  constexpr int V = P * NT;
  constexpr int IPT = ITEM / NT;
  uint64_t *tkey = reinterpret_cast<uint64_t *>(bk_raw);
  unsigned *cnt = reinterpret_cast<unsigned *>(tkey + ITEM);
  unsigned *run = cnt + V;
  int32_t *tcol = reinterpret_cast<int32_t *>(run + V);
  uint16_t *trow = reinterpret_cast<uint16_t *>(tcol + ITEM);
  for (int i = threadIdx.x; i < V; i += NT) cnt[i] = 0;
  __syncthreads();
  const long long T = item_start[nb];
  const uint32_t lmask = (uint32_t)V - 1u;
  uint2 x[IPT];
  uint64_t kv[IPT];
  int64_t lo = 0, hi = 0, bs = 0;
  int b = 0;
  auto load_item = [&](long long it) {
    b = item_range(item_start, imap, nb, O, nblk, nnz, ITEM, it, &lo, &hi, &bs);
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int64_t i = lo + threadIdx.x + (int64_t)k * NT;
      x[k] = i < hi ? rec_load<PACK>(rc, i, S) : make_uint2(NOREC, 0);
      kv[k] = i < hi ? __ldcs(rkey + i) : 0ull;
    }
  };
  // over sub-buckets (P = 1), the item after the next one is asked into L2
  // while this one is written out (the next one is loaded into registers
  // then): R-MAT 26 placement 16.1 -> 15.5 ms; over the wider buckets it
  // measured slower (R-MAT 20 323 -> 331 us), and so did the degree pass
  auto prefetch_item = [&](long long it2) {
    if (P != 1 || threadIdx.x != 0 || it2 >= T) return;
    int64_t l2, h2, b2;
    item_range(item_start, imap, nb, O, nblk, nnz, ITEM, it2, &l2, &h2, &b2);
    const int64_t tot = *nnz;
    l2_prefetch(rc, PACK ? 4 : 8, l2, h2, tot);
    l2_prefetch(rkey, 8, l2, h2, tot);
  };
  if ((long long)blockIdx.x < T) load_item(blockIdx.x);
  prefetch_item((long long)blockIdx.x + gridDim.x);
  for (long long it = blockIdx.x; it < T; it += gridDim.x) {
    const int64_t v0 = (int64_t)b << S, ibs = bs;
    unsigned rk[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k)
      if (x[k].x != NOREC) rk[k] = atomicAdd(cnt + (x[k].x & lmask), 1u);
    __syncthreads();
    // claims by the counter owners (in row order); their results are stored
    // after the sort so that the atomics overlap it
    unsigned long long claim[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int j = threadIdx.x * P + k;
      const unsigned c = cnt[j];
      claim[k] = (c && v0 + j < n) ? atomicAdd(cursor + v0 + j, (unsigned long long)c) : 0ull;
    }
    const unsigned total = block_scan_excl<NT>(cnt, V);  // cnt[j] = start of row j in the sorted item
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (x[k].x == NOREC) continue;
      const unsigned lr = x[k].x & lmask;
      const unsigned sp = cnt[lr] + rk[k];
      trow[sp] = (uint16_t)lr;
      tcol[sp] = (int32_t)x[k].y;
      tkey[sp] = kv[k];
    }
    // the next item's records are loaded while this one is written out
    prefetch_item(it + 2 * (long long)gridDim.x);
    if (it + gridDim.x < T) load_item(it + gridDim.x);
#pragma unroll
    for (int k = 0; k < P; ++k) run[threadIdx.x * P + k] = (unsigned)(claim[k] - (unsigned long long)ibs);
    __syncthreads();
    for (unsigned sp = threadIdx.x; sp < total; sp += NT) {
      const unsigned lr = trow[sp];
      const int64_t pos = ibs + run[lr] + (sp - cnt[lr]);
      col[pos] = tcol[sp];
      key[pos] = tkey[sp];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < V; i += NT) cnt[i] = 0;
    __syncthreads();
  }
}

// ---- two-level buckets (more than VMAX rows per bucket: large graphs) -------------
// With 2^S > VMAX rows per bucket, the records of an item mostly belong to
// different rows, and claiming slots row by row would cost one global atomic
// per record.  A second partition splits every bucket into sub-buckets of
// 2^SUBS rows: chunks of one bucket's records count their records per
// sub-bucket (pass 2a); an exclusive scan of the counts in (bucket,
// sub-bucket, chunk) order gives every chunk a place in every sub-bucket; the
// chunk then writes each tile of its records sorted by sub-bucket, one
// contiguous run per (tile, sub-bucket) (pass 2b).  The records are then
// grouped by row >> SUBS in row order, and the item passes 3 and 5 run over
// the sub-buckets with direct shared-memory counters: an item of ITEM5
// records meets at most 2^SUBS rows, so it claims at most that many runs.
constexpr int SUBS = 9;                // rows per sub-bucket: 2^SUBS (P = 1 in pass 5)
constexpr int CH2 = 65536;             // records per chunk of pass 2
constexpr int TR2 = 4096;              // records per tile of pass 2
constexpr int RPT2 = TR2 / BT2;        // records per thread and tile
constexpr int NSMAX = 4096;            // sub-buckets per bucket at most (S <= 21)
constexpr int CNT_UNR = 8;             // records per thread and step of pass 2a

// Pass 2a: H2[c0 * NS + d * nch + c] = records of sub-bucket d in chunk c of
// bucket b (c0 = its first chunk, nch = its chunks).
__global__ void __launch_bounds__(BT) k_sb_count(const long long *chunk_start, const int *imap, int nb,
                                                 const long long *O,
                                                 int nblk, const long long *nnz, const uint2 *__restrict__ rc,
                                                 int NS, long long *H2) {
  __shared__ unsigned cnt[NSMAX];
  const long long T = chunk_start[nb];
  const uint32_t dmask = (uint32_t)NS - 1u;
  for (long long it = blockIdx.x; it < T; it += gridDim.x) {
    for (int i = threadIdx.x; i < NS; i += BT) cnt[i] = 0;
    __syncthreads();
    int64_t lo, hi, bs;
    const int b = item_range(chunk_start, imap, nb, O, nblk, nnz, CH2, it, &lo, &hi, &bs);
    for (int64_t i0 = lo; i0 < hi; i0 += CNT_UNR * BT) {
      // CNT_UNR loads in flight per thread before the first count
      uint32_t d[CNT_UNR];
#pragma unroll
      for (int k = 0; k < CNT_UNR; ++k) {
        const int64_t i = i0 + threadIdx.x + (int64_t)k * BT;
        d[k] = i < hi ? ((__ldcs(&rc[i].x) >> SUBS) & dmask) : NOREC;
      }
#pragma unroll
      for (int k = 0; k < CNT_UNR; ++k)
        if (d[k] != NOREC) atomicAdd(cnt + d[k], 1u);
    }
    __syncthreads();
    const long long c0 = chunk_start[b], nch = chunk_start[b + 1] - c0, cl = it - c0;
    for (int d = threadIdx.x; d < NS; d += BT) H2[c0 * NS + (long long)d * nch + cl] = cnt[d];
    __syncthreads();
  }
}

__global__ void k_sb_len(const long long *chunk_start, int nb, int NS, long long *len) {
  *len = chunk_start[nb] * NS;
}

// Shared memory of pass 2b: the tile sorted by sub-bucket (row, column, key),
// then per sub-bucket the running global position (u64), the count and the
// run start (u32 each; nsp = NS rounded up to BT2).
__host__ __device__ constexpr size_t sb_scatter_smem(int nsp) { return (size_t)TR2 * 16 + (size_t)nsp * 16; }

// Pass 2b.  H2 scanned: chunk c of bucket b writes its records of sub-bucket
// d to [H2[c0 * NS + d * nch + c], ...), one run per (tile, sub-bucket).
__global__ void __launch_bounds__(BT2) k_sb_scatter(const long long *chunk_start, const int *imap, int nb,
                                                   const long long *O,
                                                   int nblk, const long long *nnz, const uint2 *__restrict__ rc,
                                                   const uint64_t *__restrict__ rkey, int NS, int nsp,
                                                   const long long *__restrict__ H2, uint2 *__restrict__ rc2,
                                                   uint64_t *__restrict__ rkey2) {
  extern __shared__ __align__(16) unsigned char sb_raw[];
  uint4 *tile = reinterpret_cast<uint4 *>(sb_raw);  // (row, col, key low, key high)
  unsigned long long *gbase = reinterpret_cast<unsigned long long *>(tile + TR2);
  unsigned *cnt = reinterpret_cast<unsigned *>(gbase + nsp);
  unsigned *start = cnt + nsp;
  const long long T = chunk_start[nb];
  const uint32_t dmask = (uint32_t)NS - 1u;
  for (int i = threadIdx.x; i < nsp; i += BT2) cnt[i] = 0;
  for (long long it = blockIdx.x; it < T; it += gridDim.x) {
    int64_t lo, hi, bs;
    const int b = item_range(chunk_start, imap, nb, O, nblk, nnz, CH2, it, &lo, &hi, &bs);
    const long long c0 = chunk_start[b], nch = chunk_start[b + 1] - c0, cl = it - c0;
    for (int d = threadIdx.x; d < nsp; d += BT2)
      gbase[d] = d < NS ? (unsigned long long)H2[c0 * NS + (long long)d * nch + cl] : 0ull;
    __syncthreads();
    for (int64_t t0 = lo; t0 < hi; t0 += TR2) {
      // the next tile's records are asked into L2 while this one is sorted
      // (the block's next chunk's first tile after its last)
      if (threadIdx.x == 0) {
        int64_t n0 = t0 + TR2, n1 = hi, nb2;
        if (n0 >= hi && it + gridDim.x < T) item_range(chunk_start, imap, nb, O, nblk, nnz, CH2, it + gridDim.x, &n0, &n1, &nb2);
        if (n0 < n1) {
          const int64_t e1 = min64(n0 + TR2, n1), tot = *nnz;
          l2_prefetch(rc, 8, n0, e1, tot);
          l2_prefetch(rkey, 8, n0, e1, tot);
        }
      }
      uint2 x[RPT2];
      uint64_t kv[RPT2];
      unsigned rk[RPT2];
#pragma unroll
      for (int k = 0; k < RPT2; ++k) {
        const int64_t i = t0 + threadIdx.x + (int64_t)k * BT2;
        x[k] = i < hi ? __ldcs(rc + i) : make_uint2(NOREC, 0);
        kv[k] = i < hi ? __ldcs(rkey + i) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < RPT2; ++k)
        if (x[k].x != NOREC) rk[k] = atomicAdd(cnt + ((x[k].x >> SUBS) & dmask), 1u);
      __syncthreads();
      for (int i = threadIdx.x; i < nsp; i += BT2) start[i] = cnt[i];
      __syncthreads();
      const unsigned total = block_scan_excl<BT2>(start, nsp);
#pragma unroll
      for (int k = 0; k < RPT2; ++k) {
        if (x[k].x == NOREC) continue;
        const uint32_t d = (x[k].x >> SUBS) & dmask;
        tile[start[d] + rk[k]] = make_uint4(x[k].x, x[k].y, (uint32_t)kv[k], (uint32_t)(kv[k] >> 32));
      }
      __syncthreads();
      for (unsigned i = threadIdx.x; i < total; i += BT2) {
        const uint4 y = tile[i];
        const uint32_t d = (y.x >> SUBS) & dmask;
        const unsigned long long pos = gbase[d] + (i - start[d]);
        rc2[pos] = make_uint2(y.x, y.y);
        rkey2[pos] = ((uint64_t)y.w << 32) | y.z;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nsp; i += BT2) {
        gbase[i] += cnt[i];
        cnt[i] = 0;
      }
      __syncthreads();
    }
  }
}

// First record of every sub-bucket g = b * NS + d: the scanned H2 at the
// bucket's first chunk (an empty bucket has no chunks: its start).
__global__ void __launch_bounds__(BT) k_sb_starts(const long long *chunk_start, int nb, const long long *O,
                                                  int nblk, int NS, const long long *H2, long long *sub_start) {
  const int64_t NSUB = (int64_t)nb * NS;
  for (int64_t g = (int64_t)blockIdx.x * BT + threadIdx.x; g < NSUB; g += (int64_t)gridDim.x * BT) {
    const int b = (int)(g / NS), d = (int)(g % NS);
    const long long c0 = chunk_start[b], nch = chunk_start[b + 1] - c0;
    sub_start[g] = nch > 0 ? H2[c0 * NS + (long long)d * nch] : O[(int64_t)b * nblk];
  }
}


int ceil_log2(int64_t n) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << b) < n) ++b;
  return b;
}

}  // namespace

bool bucket_build_fits(int64_t n) { return n <= ((int64_t)1 << 31); }

int bucket_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *w, int wtype,
                     int32_t G, const int64_t *eoff_d, const int64_t *voff_d, int2 *ends, long long *small,
                     CsrBuf &csr, cudaStream_t s) {
  if (!bucket_build_fits(n)) return fail(MSF_ERR_TOO_LARGE, "bucketed CSR builder: too many vertices");
  int err = MSF_OK;
  void *keep[20] = {nullptr};
  int nk = 0;
  auto get = [&](size_t bytes) -> void * {
    void *q = err ? nullptr : pool_alloc(bytes, &err);
    if (q) keep[nk++] = q;
    return q;
  };
  auto release = [&]() {  // behind the work queued on s
    for (int i = 0; i < nk; ++i) pool_free_after(keep[i], s);
  };
  // 2^S vertices per bucket: at least 2048 (fewer, longer runs per bucket in
  // pass 2), at most NBMAX buckets (runs of pass 2); beyond 2^12 rows per
  // bucket the buckets are split again into sub-buckets of 2^SUBS rows
  int S = ceil_log2(n) - 10;
  if (S < 11) S = 11;
  const int nb = (int)((n + ((int64_t)1 << S) - 1) >> S) > 0 ? (int)((n + ((int64_t)1 << S) - 1) >> S) : 1;
  const int nbp = (nb + BT1 - 1) / BT1 * BT1;
  const size_t smem_scatter = scatter_smem(nbp);
  const bool wide = S > 12;  // more rows per bucket than the item passes can count directly
  const int NS = wide ? 1 << (S - SUBS) : 1;  // sub-buckets per bucket
  const int nsp = (NS + BT2 - 1) / BT2 * BT2;
  const int S3 = wide ? SUBS : S;              // rows per group of the item passes: 2^S3
  const int ng = wide ? nb * NS : nb;          // groups of the item passes
  const int item5 = wide ? ITEM5 : ITEM5N;  // records per item of pass 5
  const size_t smem_place = place_smem(1 << S3, item5);
  const int nblk = sm_count() * 2;  // edge chunks of passes 1 and 2
  int64_t E = (m + nblk - 1) / nblk;
  E = (E + 3) / 4 * 4;  // whole quads of edges per block (16-byte loads in the validation)
  if (E < 4) E = 4;
  const int64_t cap = 2 * m > 0 ? 2 * m : 1;
  // one-word records when the column fits beside the bucket-local row
  const bool pack = !wide && ceil_log2(n) + S <= 32;
  void *rc = get((size_t)cap * (pack ? sizeof(uint32_t) : sizeof(uint2)));
  uint64_t *rkey = (uint64_t *)get((size_t)cap * sizeof(uint64_t));
  long long *H = (long long *)get((size_t)nb * nblk * sizeof(long long));
  long long *items3 = (long long *)get((size_t)(ng + 1) * sizeof(long long));
  long long *items5 = (long long *)get((size_t)(ng + 1) * sizeof(long long));
  int64_t *scan_tmp = (int64_t *)get((size_t)(NB_SCAN + 1) * 8);
  long long *sm = (long long *)get(64);  // [0] histogram length, [1] records, [2] sub-bucket histogram length,
                                         // [3] groups of the item passes (sub-bucket path)
  unsigned *deg = (unsigned *)get((size_t)(n + 1) * sizeof(unsigned));
  int64_t *cursor = (int64_t *)get((size_t)(n + 1) * sizeof(int64_t));
  // second level: chunks of pass 2, their sub-bucket counts, the regrouped
  // records and the sub-bucket starts
  const int64_t max_chunks = (cap + CH2 - 1) / CH2 + nb;
  long long *chunks = wide ? (long long *)get((size_t)(nb + 1) * sizeof(long long)) : nullptr;
  long long *H2 = wide ? (long long *)get((size_t)max_chunks * NS * sizeof(long long)) : nullptr;
  uint2 *rc2 = wide ? (uint2 *)get((size_t)cap * sizeof(uint2)) : nullptr;
  uint64_t *rkey2 = wide ? (uint64_t *)get((size_t)cap * sizeof(uint64_t)) : nullptr;
  long long *sub_start = wide ? (long long *)get((size_t)(ng + 1) * sizeof(long long)) : nullptr;
  // item -> bucket maps (the items of a bucket, or of a sub-bucket, or the chunks)
  int *imap3 = (int *)get((size_t)((cap + ITEM3 - 1) / ITEM3 + ng + 1) * sizeof(int));
  int *imap5 = (int *)get((size_t)((cap + item5 - 1) / item5 + ng + 1) * sizeof(int));
  int *cmap = wide ? (int *)get((size_t)max_chunks * sizeof(int)) : nullptr;
  if (err) {
    release();
    return err;
  }
  cudaFuncSetAttribute(k_bk_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_scatter);
  cudaFuncSetAttribute(k_bk_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_scatter);
  cudaFuncSetAttribute(k_sb_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb_scatter_smem(nsp));
  cudaFuncSetAttribute(k_bk_place<1, false, BT5, ITEM5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_place);
  cudaFuncSetAttribute(k_bk_place<2, true, BT5N, ITEM5N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_place);
  cudaFuncSetAttribute(k_bk_place<2, false, BT5N, ITEM5N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_place);
  cudaFuncSetAttribute(k_bk_place<4, false, BT5N, ITEM5N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_place);
  const int item_grid = sm_count() * 4;

  cudaError_t e = cudaMemsetAsync(deg, 0, (size_t)(n + 1) * sizeof(unsigned), s);
  {
    int *errw = (int *)(small + 3);
    auto *nl = (unsigned long long *)(small + 5);
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    if (vec)
      k_bk_validate<true><<<nblk, BTV, 0, s>>>(src, dst, wtype, m, n, G, eoff_d, voff_d, E, nb, S, ends, errw, nl, H, sm);
    else
      k_bk_validate<false><<<nblk, BTV, 0, s>>>(src, dst, wtype, m, n, G, eoff_d, voff_d, E, nb, S, ends, errw, nl, H, sm);
  }
  launch_scan_excl(reinterpret_cast<int64_t *>(H), reinterpret_cast<int64_t *>(H),
                   reinterpret_cast<const int64_t *>(sm), scan_tmp, reinterpret_cast<int64_t *>(sm + 1), s);
  if (pack)
    k_bk_scatter<true><<<nblk, BT1, smem_scatter, s>>>(ends, w, wtype, m, E, nb, nbp, S, H, rc, rkey,
                                                       (int *)(small + 3));
  else
    k_bk_scatter<false><<<nblk, BT1, smem_scatter, s>>>(ends, w, wtype, m, E, nb, nbp, S, H, rc, rkey,
                                                        (int *)(small + 3));
  // the groups of the item passes: the buckets, or the sub-buckets
  const long long *GO = H;  // group g starts at GO[g * gstride]
  int gstride = nblk;
  const void *grc = rc;
  const uint64_t *gkey = rkey;
  if (wide) {
    k_bk_items<<<1, 1024, 0, s>>>(H, nb, nblk, sm + 1, CH2, chunks, 0, nullptr);
    k_bk_item_map<<<sm_count() * 4, BT, 0, s>>>(chunks, nb, cmap, nullptr, nullptr);
    k_sb_count<<<item_grid, BT, 0, s>>>(chunks, cmap, nb, H, nblk, sm + 1, (const uint2 *)rc, NS, H2);
    k_sb_len<<<1, 1, 0, s>>>(chunks, nb, NS, sm + 2);
    launch_scan_excl(reinterpret_cast<int64_t *>(H2), reinterpret_cast<int64_t *>(H2),
                     reinterpret_cast<const int64_t *>(sm + 2), scan_tmp, nullptr, s);
    k_sb_scatter<<<sm_count() * 2, BT2, sb_scatter_smem(nsp), s>>>(chunks, cmap, nb, H, nblk, sm + 1, (const uint2 *)rc,
                                                                  rkey, NS, nsp, H2, rc2, rkey2);
    k_sb_starts<<<sm_count() * 4, BT, 0, s>>>(chunks, nb, H, nblk, NS, H2, sub_start);
    GO = sub_start;
    gstride = 1;
    grc = rc2;
    gkey = rkey2;
  }
  if (wide) {
    // many groups: counts on every SM, then a scan of each list (sm[3]: ng)
    static_assert((ITEM3 & (ITEM3 - 1)) == 0 && (ITEM5 & (ITEM5 - 1)) == 0, "item sizes are powers of two");
    k_bk_counts<<<sm_count() * 4, BT, 0, s>>>(GO, ng, gstride, sm + 1, ceil_log2(ITEM3), items3, ceil_log2(item5),
                                              items5, sm + 3);
    launch_scan_excl(reinterpret_cast<int64_t *>(items3), reinterpret_cast<int64_t *>(items3),
                     reinterpret_cast<const int64_t *>(sm + 3), scan_tmp, reinterpret_cast<int64_t *>(items3 + ng), s);
    launch_scan_excl(reinterpret_cast<int64_t *>(items5), reinterpret_cast<int64_t *>(items5),
                     reinterpret_cast<const int64_t *>(sm + 3), scan_tmp, reinterpret_cast<int64_t *>(items5 + ng), s);
  } else {
    k_bk_items<<<1, 1024, 0, s>>>(GO, ng, gstride, sm + 1, ITEM3, items3, item5, items5);
  }
  k_bk_item_map<<<sm_count() * 4, BT, 0, s>>>(items3, ng, imap3, items5, imap5);
  if (pack)
    k_bk_degree<true><<<item_grid, BT, 0, s>>>(items3, imap3, ng, GO, gstride, sm + 1, grc, S3, n, deg);
  else
    k_bk_degree<false><<<item_grid, BT, 0, s>>>(items3, imap3, ng, GO, gstride, sm + 1, grc, S3, n, deg);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "bucketed CSR build");
  }
  if (int rc_ = rows_from_degrees(n, deg, small, csr, cursor, s)) {
    release();
    return rc_;
  }
  auto *cur = reinterpret_cast<unsigned long long *>(cursor);
  const int place_grid = sm_count() * 2;
  if (S3 == SUBS)
    k_bk_place<1, false, BT5, ITEM5><<<place_grid, BT5, smem_place, s>>>(items5, imap5, ng, GO, gstride, sm + 1, grc,
                                                                         gkey, S3, n, cur, csr.col, csr.key);
  else if (S3 == 11 && pack)
    k_bk_place<2, true, BT5N, ITEM5N><<<sm_count(), BT5N, smem_place, s>>>(items5, imap5, ng, GO, gstride, sm + 1,
                                                                           grc, gkey, S3, n, cur, csr.col, csr.key);
  else if (S3 == 11)
    k_bk_place<2, false, BT5N, ITEM5N><<<sm_count(), BT5N, smem_place, s>>>(items5, imap5, ng, GO, gstride, sm + 1,
                                                                            grc, gkey, S3, n, cur, csr.col, csr.key);
  else
    k_bk_place<4, false, BT5N, ITEM5N><<<sm_count(), BT5N, smem_place, s>>>(items5, imap5, ng, GO, gstride, sm + 1,
                                                                            grc, gkey, S3, n, cur, csr.col, csr.key);
  e = cudaGetLastError();
  release();
  if (e != cudaSuccess) return cuda_fail(e, "bucketed CSR build");
  return MSF_OK;
}

}  // namespace msf

// CSR build: stable LSD radix grouping of the directed slots by row.
//
// Every non-loop edge e = (u, v) gives two slots (row u, col v) and (row v,
// col u) with the key ord(w_e) << 32 | e.  Grouping the slots by row with a
// stable least-significant-digit radix sort (digits of at most 10 bits) puts
// every row's slots together without global atomics: each pass is
//   upsweep    per-block digit histogram of a contiguous chunk (shared memory,
//              warp-aggregated counts),
//   scan       of the histograms in (digit, block) order (global offsets),
//   downsweep  the block re-reads its chunk in sub-tiles of 4096 slots staged
//              in shared memory, ranks each slot stably among equal digits
//              (__match_any_sync per 32 slots, per-warp counters) and writes
//              it to its final place of the pass.
// The first pass reads the edges (endpoint table and weights) and makes the
// slots; the last pass writes the CSR's column and key arrays and the sorted
// rows, from which the row boundaries are taken.  Within a row the slots
// keep the order of the input (edge, direction), so the CSR is deterministic.
#include "internal.cuh"

namespace msf {

namespace {

constexpr int RT = 256;                  // threads per block
constexpr int RW = RT / 32;              // warps per block
constexpr int SUB = 4096;                // slots per sub-tile (16 per thread)
constexpr int SUB_E = SUB / 2;           // edges per sub-tile in the first pass
constexpr int MAXB = 1024;               // bins per pass at most
constexpr uint32_t NOROW = 0xffffffffu;  // an empty place of a sub-tile
constexpr unsigned FULL = 0xffffffffu;

struct DownSmem {
  uint4 tile[SUB];              // x = row, y = col, z/w = key (low, high)
  uint32_t wcnt[RW][MAXB];      // per-warp counts, then per-warp offsets
  uint32_t lstart[MAXB];        // start of each digit in the locally sorted sub-tile
  uint32_t subtot[MAXB];        // slots per digit in the sub-tile
  long long boff[MAXB];         // running output position per digit
  uint32_t part[RT];            // block scan partials
};

__device__ __forceinline__ int64_t chunk_size(int64_t n_in, int quantum) {
  int64_t c = (n_in + gridDim.x - 1) / gridDim.x;
  return (c + quantum - 1) / quantum * quantum;
}

__device__ __forceinline__ uint4 make_slot(uint32_t row, uint32_t col, uint64_t key) {
  return make_uint4(row, col, (uint32_t)key, (uint32_t)(key >> 32));
}

// Number of input elements of this pass: edges (first pass) or slots.
__device__ __forceinline__ int64_t pass_len(bool edges, int64_t m, const long long *nslots) {
  return edges ? m : (int64_t)*nslots;
}

template <bool EDGES>
__global__ void __launch_bounds__(RT) k_rs_up(const int2 *ends, const uint32_t *w, int64_t m, const uint4 *slots,
                                              const long long *nslots, int shift, int bins, long long *hist) {
  __shared__ unsigned int cnt[MAXB];
  for (int i = threadIdx.x; i < bins; i += RT) cnt[i] = 0;
  __syncthreads();
  const int64_t n_in = pass_len(EDGES, m, nslots);
  const int64_t C = chunk_size(n_in, EDGES ? SUB_E : SUB);
  const int64_t lo = (int64_t)blockIdx.x * C;
  const int64_t hi = lo + C < n_in ? lo + C : n_in;
  const uint32_t dmask = (uint32_t)bins - 1u;
  const int lane = threadIdx.x & 31;
  for (int64_t base = lo; base < hi; base += RT) {
    const int64_t i = base + threadIdx.x;
    int d0 = bins, d1 = bins;
    if (i < hi) {
      if (EDGES) {
        const int2 uv = ends[i];
        if (uv.x != uv.y) {
          d0 = (int)(((uint32_t)uv.x >> shift) & dmask);
          d1 = (int)(((uint32_t)uv.y >> shift) & dmask);
        }
      } else {
        d0 = (int)((slots[i].x >> shift) & dmask);
      }
    }
    unsigned peers = __match_any_sync(FULL, d0);
    if (d0 < bins && lane == __ffs(peers) - 1) atomicAdd(&cnt[d0], (unsigned)__popc(peers));
    if (EDGES) {
      peers = __match_any_sync(FULL, d1);
      if (d1 < bins && lane == __ffs(peers) - 1) atomicAdd(&cnt[d1], (unsigned)__popc(peers));
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < bins; b += RT) hist[(int64_t)b * gridDim.x + blockIdx.x] = cnt[b];
}

template <bool EDGES, bool FINAL>
__global__ void __launch_bounds__(RT, 2) k_rs_down(const int2 *ends, const uint32_t *w, int wtype, int64_t m,
                                                const uint4 *slots, const long long *nslots, int shift, int bins,
                                                const long long *offs, uint4 *out, int32_t *out_col,
                                                uint64_t *out_key, int32_t *out_row) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DownSmem &sm = *reinterpret_cast<DownSmem *>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t n_in = pass_len(EDGES, m, nslots);
  const int64_t C = chunk_size(n_in, EDGES ? SUB_E : SUB);
  const int64_t lo = (int64_t)blockIdx.x * C;
  const int64_t hi = lo + C < n_in ? lo + C : n_in;
  const uint32_t dmask = (uint32_t)bins - 1u;
  for (int b = threadIdx.x; b < bins; b += RT) sm.boff[b] = offs[(int64_t)b * gridDim.x + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;

  constexpr int PER = SUB / RT;   // slots per thread (16)
  constexpr int BPT = MAXB / RT;  // digits per thread in the block scans (4)
  for (int64_t sub = lo; sub < hi; sub += (EDGES ? SUB_E : SUB)) {
    // stage the sub-tile (coalesced reads; the first pass makes two slots per edge)
    if (EDGES) {
      for (int k = threadIdx.x; k < SUB_E; k += RT) {
        const int64_t e = sub + k;
        uint4 a = make_uint4(NOROW, 0, 0, 0), b = a;
        if (e < hi) {
          const int2 uv = ends[e];
          if (uv.x != uv.y) {
            const uint64_t key = ((uint64_t)ord_weight_dev(w[e], wtype) << 32) | (uint64_t)e;
            a = make_slot((uint32_t)uv.x, (uint32_t)uv.y, key);
            b = make_slot((uint32_t)uv.y, (uint32_t)uv.x, key);
          }
        }
        sm.tile[2 * k] = a;
        sm.tile[2 * k + 1] = b;
      }
    } else {
      for (int k = threadIdx.x; k < SUB; k += RT) {
        const int64_t i = sub + k;
        sm.tile[k] = i < hi ? slots[i] : make_uint4(NOROW, 0, 0, 0);
      }
    }
    for (int i = threadIdx.x; i < RW * MAXB; i += RT) (&sm.wcnt[0][0])[i] = 0;
    __syncthreads();
    // rank: each warp walks its 512 places in order; a slot's place among the
    // warp's slots of its digit = count before this step + rank in the step
    uint4 it[PER];
    int dg[PER];
    uint32_t wl[PER];
#pragma unroll
    for (int step = 0; step < PER; ++step) {
      it[step] = sm.tile[wid * (SUB / RW) + step * 32 + lane];
      dg[step] = it[step].x == NOROW ? bins : (int)((it[step].x >> shift) & dmask);
      const unsigned peers = __match_any_sync(FULL, dg[step]);
      const bool ok = dg[step] < bins;
      wl[step] = (ok ? sm.wcnt[wid][dg[step]] : 0u) + __popc(peers & lt);
      __syncwarp();
      if (ok && lane == __ffs(peers) - 1) sm.wcnt[wid][dg[step]] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per-warp bases within each digit, digit totals, and the digit starts of
    // the locally sorted sub-tile (block exclusive scan over the digits)
    uint32_t mysum = 0;
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int b = threadIdx.x * BPT + q;
      uint32_t run = 0;
      if (b < bins) {
        for (int x = 0; x < RW; ++x) {
          const uint32_t t = sm.wcnt[x][b];
          sm.wcnt[x][b] = run;
          run += t;
        }
      }
      sm.subtot[b] = run;
      mysum += run;
    }
    sm.part[threadIdx.x] = mysum;
    __syncthreads();
    if (wid == 0) {
      uint32_t acc = 0;
      for (int x = lane * (RT / 32); x < (lane + 1) * (RT / 32); ++x) acc += sm.part[x];
      uint32_t incl = acc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
      }
      uint32_t run = incl - acc;
      for (int x = lane * (RT / 32); x < (lane + 1) * (RT / 32); ++x) {
        const uint32_t t = sm.part[x];
        sm.part[x] = run;
        run += t;
      }
    }
    __syncthreads();
    {
      uint32_t run = sm.part[threadIdx.x];
#pragma unroll
      for (int q = 0; q < BPT; ++q) {
        const int b = threadIdx.x * BPT + q;
        sm.lstart[b] = run;
        run += sm.subtot[b];
      }
    }
    __syncthreads();
    // local sort of the sub-tile by digit (stable), in place
#pragma unroll
    for (int step = 0; step < PER; ++step) {
      if (dg[step] < bins) sm.tile[sm.lstart[dg[step]] + sm.wcnt[wid][dg[step]] + wl[step]] = it[step];
    }
    __syncthreads();
    // coalesced write of the digit runs
    uint32_t nvalid = 0;
    {
      uint32_t v = 0;
#pragma unroll
      for (int q = 0; q < BPT; ++q) v += sm.subtot[threadIdx.x * BPT + q];
      // total valid slots of the sub-tile = last digit start + its count
      nvalid = sm.lstart[MAXB - 1] + sm.subtot[MAXB - 1];
      (void)v;
    }
    for (int k = threadIdx.x; k < (int)nvalid; k += RT) {
      const uint4 x = sm.tile[k];
      const int d = (int)((x.x >> shift) & dmask);
      const int64_t dest = sm.boff[d] + (k - (int)sm.lstart[d]);
      if (FINAL) {
        out_col[dest] = (int32_t)x.y;
        out_key[dest] = ((uint64_t)x.w << 32) | x.z;
        out_row[dest] = (int32_t)x.x;
      } else {
        out[dest] = x;
      }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < bins; b += RT) sm.boff[b] += sm.subtot[b];
    __syncthreads();
  }
}

// Row boundaries of the sorted rows: a slot starts a row when its row differs
// from its predecessor's.  Count per block chunk, scan, then write rows[] and
// rp[] in order.
__global__ void __launch_bounds__(RT) k_rb_count(const int32_t *row, const long long *nslots, long long *bcount) {
  const int64_t n = *nslots;
  const int64_t C = chunk_size(n, RT);
  const int64_t lo = (int64_t)blockIdx.x * C, hi = lo + C < n ? lo + C : n;
  unsigned cnt = 0;
  for (int64_t s = lo + threadIdx.x; s < hi; s += RT) cnt += (s == 0 || row[s] != row[s - 1]);
  __shared__ unsigned tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) cnt += __shfl_xor_sync(FULL, cnt, d);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&tot, cnt);
  __syncthreads();
  if (threadIdx.x == 0) bcount[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(RT) k_rb_write(const int32_t *row, const long long *nslots, const long long *boffs,
                                                 const long long *nrows, int32_t *rows, int64_t *rp) {
  const int64_t n = *nslots;
  const int64_t C = chunk_size(n, RT);
  const int64_t lo = (int64_t)blockIdx.x * C, hi = lo + C < n ? lo + C : n;
  __shared__ long long run;
  if (threadIdx.x == 0) run = boffs[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ unsigned wsum[RW];
  for (int64_t base = lo; base < hi; base += RT) {
    const int64_t s = base + threadIdx.x;
    const bool head = s < hi && (s == 0 || row[s] != row[s - 1]);
    const unsigned bal = __ballot_sync(FULL, head);
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int q = 0; q < RW; ++q) {
      before += (q < wid) ? wsum[q] : 0;
      all += wsum[q];
    }
    if (head) {
      const int64_t k = run + before + __popc(bal & ((1u << lane) - 1u));
      rows[k] = row[s];
      rp[k] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) run += all;
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rp[*nrows] = n;
}

__global__ void k_set(long long *a, long long v) { *a = v; }

}  // namespace

// Groups the 2 * (non-loop edges) slots by row into csr (col, key, rows, rp)
// from the validated endpoint table.  nslots_dev holds the slot count (twice
// the number of non-loop edges); the row count is written to *nrows_dev.
int radix_build_csr(int64_t n, int64_t m, const int2 *ends, const uint32_t *w, int wtype,
                    const long long *nslots_dev, long long *nrows_dev, CsrBuf &csr, cudaStream_t s) {
  int err = MSF_OK;
  const int NB = sm_count() * 2;
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;  // rows < n <= 2^bits
  const int passes = bits <= 10 ? 1 : (bits + 9) / 10;
  const int db = bits == 0 ? 1 : (bits + passes - 1) / passes;
  const int bins = 1 << db;
  const size_t smem = sizeof(DownSmem);
  // scratch
  void *keep[6] = {nullptr};
  int nk = 0;
  auto get = [&](size_t bytes) -> void * {
    void *q = pool_alloc(bytes, &err);
    keep[nk++] = q;
    return q;
  };
  const int64_t cap = 2 * m > 0 ? 2 * m : 1;
  uint4 *bufA = passes >= 2 ? (uint4 *)get((size_t)cap * sizeof(uint4)) : nullptr;
  uint4 *bufB = (!err && passes >= 3) ? (uint4 *)get((size_t)cap * sizeof(uint4)) : nullptr;
  int32_t *rowtmp = err ? nullptr : (int32_t *)get((size_t)cap * sizeof(int32_t));
  long long *hist = err ? nullptr : (long long *)get((size_t)(MAXB * NB + 16) * sizeof(long long));
  long long *scratch = err ? nullptr : (long long *)get((size_t)(NB_SCAN + 64) * sizeof(long long));
  long long *small = err ? nullptr : (long long *)get(64);
  if (err) {
    for (int i = 0; i < nk; ++i) pool_free(keep[i]);
    return err;
  }
  cudaFuncSetAttribute(k_rs_down<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_rs_down<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_rs_down<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_rs_down<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  long long *nbins = small;  // histogram length for the scan
  k_set<<<1, 1, 0, s>>>(nbins, (long long)bins * NB);
  const uint4 *in = nullptr;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * db;
    const bool first = p == 0, last = p == passes - 1;
    uint4 *outb = (p % 2 == 0) ? bufA : bufB;
    if (first)
      k_rs_up<true><<<NB, RT, 0, s>>>(ends, w, m, nullptr, nslots_dev, shift, bins, hist);
    else
      k_rs_up<false><<<NB, RT, 0, s>>>(nullptr, nullptr, m, in, nslots_dev, shift, bins, hist);
    launch_scan_excl(reinterpret_cast<int64_t *>(hist), reinterpret_cast<int64_t *>(hist),
                     reinterpret_cast<const int64_t *>(nbins), reinterpret_cast<int64_t *>(scratch), nullptr, s);
    if (first && last)
      k_rs_down<true, true><<<NB, RT, smem, s>>>(ends, w, wtype, m, nullptr, nslots_dev, shift, bins, hist, nullptr,
                                                 csr.col, csr.key, rowtmp);
    else if (first)
      k_rs_down<true, false><<<NB, RT, smem, s>>>(ends, w, wtype, m, nullptr, nslots_dev, shift, bins, hist, outb,
                                                  nullptr, nullptr, nullptr);
    else if (last)
      k_rs_down<false, true><<<NB, RT, smem, s>>>(nullptr, nullptr, wtype, m, in, nslots_dev, shift, bins, hist,
                                                  nullptr, csr.col, csr.key, rowtmp);
    else
      k_rs_down<false, false><<<NB, RT, smem, s>>>(nullptr, nullptr, wtype, m, in, nslots_dev, shift, bins, hist,
                                                   outb, nullptr, nullptr, nullptr);
    in = outb;
  }
  // row boundaries
  long long *nbk = small + 1;
  k_set<<<1, 1, 0, s>>>(nbk, (long long)NB);
  k_rb_count<<<NB, RT, 0, s>>>(rowtmp, nslots_dev, hist);
  launch_scan_excl(reinterpret_cast<int64_t *>(hist), reinterpret_cast<int64_t *>(hist),
                   reinterpret_cast<const int64_t *>(nbk), reinterpret_cast<int64_t *>(scratch),
                   reinterpret_cast<int64_t *>(nrows_dev), s);
  k_rb_write<<<NB, RT, 0, s>>>(rowtmp, nslots_dev, hist, nrows_dev, csr.rows, csr.rp);
  cudaError_t e = cudaGetLastError();
  // the scratch returns to the pool after the caller's synchronisation
  e = (e == cudaSuccess) ? cudaStreamSynchronize(s) : e;
  for (int i = 0; i < nk; ++i) pool_free(keep[i]);
  if (e != cudaSuccess) return cuda_fail(e, "radix CSR build");
  return MSF_OK;
}

}  // namespace msf

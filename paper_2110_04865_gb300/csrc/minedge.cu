// The multilinear min-edge kernel and the edge compaction sweeps.
//
// Multilinear function (Sec. 3.1) and projection onto the star root (the
// multilinear and projection steps of Algorithm 2):
//   q_i     = MinWeight_j f(p_i, a_ij, p_j),  f = a_ij if p_i != p_j else inf
//   r_{p_i} = MinWeight_i q_i
// With complete shortcutting every tree is a star at the start of a round
// (Sec. 4.2), so every vertex may contribute.  The value a_ij carries the
// 64-bit key ord(w) << 32 | edge id, which makes MinWeight a plain unsigned
// minimum and the result unique; the parent of the far end (the EDGE pair's
// second member) is recovered from the edge id when hooking.
//
// GPU mapping.  The slot array of the CSR is cut into tiles of S = 32 * V
// consecutive slots, one tile per warp at a time (persistent grid-stride).
// Lane l streams V columns and V keys (16-byte vector loads, evict-first),
// gathers p_j for its columns, and reads p_i from shared memory, where the
// warp staged p of every row that meets the tile.  Row starts inside the tile
// are marked in a per-warp bitmap, so each lane knows where its segments
// begin.  A lane reduces its own segments, a segmented shuffle scan joins
// segments that cross lanes, and a single atomicMin per (row, tile) segment
// writes the projection r_{p_i}.  Rows that span tiles get one atomicMin per
// tile.
//
// The same front end drives edge compaction: COUNT counts live slots
// (p_i != p_j) per tile and per row; SCATTER writes the live slots in order,
// relabelled to their current roots (components only merge, so a dead slot
// never revives).
#include "internal.cuh"

namespace msf {

namespace {

constexpr int WARPS = 8;
constexpr int THREADS = WARPS * 32;
constexpr unsigned FULL = 0xffffffffu;

enum Mode { MIN_EDGE = 0, COUNT = 1, SCATTER = 2 };

template <int V>
struct TileSmem {
  int32_t pi[WARPS][32 * V];   // p of the rows meeting the tile
  uint32_t head[WARPS][V];     // row-start bitmap, S bits
};

__device__ __forceinline__ void load_col4(const int32_t *a, int32_t *o) {
  const int4 x = __ldcs(reinterpret_cast<const int4 *>(a));
  o[0] = x.x;
  o[1] = x.y;
  o[2] = x.z;
  o[3] = x.w;
}

__device__ __forceinline__ void load_key2(const uint64_t *a, uint64_t *o) {
  const ulonglong2 x = __ldcs(reinterpret_cast<const ulonglong2 *>(a));
  o[0] = x.x;
  o[1] = x.y;
}

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}

template <int V, int MODE>
__global__ void __launch_bounds__(THREADS) k_sweep(DevState *st) {
  constexpr int S = 32 * V;
  constexpr int F = S / TB;
  __shared__ TileSmem<V> sm;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const CsrBuf B = st->buf[st->cur];
  const int64_t nnz = st->nnz, nrows = st->nrows;
  const int32_t *__restrict__ p = st->p;
  const bool ident = (MODE == MIN_EDGE) && st->first_round_identity != 0;
  unsigned long long *r = reinterpret_cast<unsigned long long *>(st->r);
  unsigned long long *rowcnt = reinterpret_cast<unsigned long long *>(st->rowcnt);
  const int64_t ntiles = (nnz + S - 1) / S;
  int32_t *s_pi = sm.pi[wid];
  uint32_t *s_head = sm.head[wid];
  CsrBuf D;
  if (MODE == SCATTER) D = st->buf[st->cur == 1 ? 2 : 1];
  unsigned long long live = 0;
  bool bad = false;

  for (int64_t t = (int64_t)blockIdx.x * WARPS + wid; t < ntiles; t += (int64_t)gridDim.x * WARPS) {
    const int64_t s0 = t * S;
    const int64_t sl = s0 + (int64_t)lane * V;
    // 1. stream the tile (independent of everything else: issue first)
    int32_t c[V];
    uint64_t k[V];
#pragma unroll
    for (int q = 0; q < V / 4; ++q) load_col4(B.col + sl + 4 * q, c + 4 * q);
    if (MODE != COUNT) {
#pragma unroll
      for (int q = 0; q < V / 2; ++q) load_key2(B.key + sl + 2 * q, k + 2 * q);
    }
    // 2. rows meeting the tile: k0 .. klast
    const int32_t k0 = B.tile_row[t * F];
    const int32_t kn = B.tile_row[(t + 1) * F];
    int32_t klast = kn;
    if (kn >= nrows || B.rp[kn] >= s0 + S) klast = kn - 1;
    int R = klast - k0 + 1;
    if (R > S) {  // impossible for a CSR without empty rows
      bad = true;
      R = S;
    }
    if (lane < V) s_head[lane] = 0u;
    __syncwarp();
    for (int idx = lane; idx < R; idx += 32) {
      const int32_t kk = k0 + idx;
      const int32_t v = B.rows[kk];
      s_pi[idx] = ident ? v : __ldg(p + v);
      if (idx > 0) {
        const int64_t pos = B.rp[kk] - s0;
        if (pos > 0 && pos < S) atomicOr(&s_head[pos >> 5], 1u << (pos & 31));
        else bad = true;
      }
    }
    // 3. p_j of the columns
    int32_t pj[V];
#pragma unroll
    for (int j = 0; j < V; ++j) pj[j] = ident ? c[j] : __ldg(p + c[j]);
    __syncwarp();
    // 4. where the lane's segments start
    const int base = lane * V;
    const int w0 = base >> 5, sh = base & 31;
    uint32_t hv = s_head[w0] >> sh;
    if (V < 32) hv &= (1u << V) - 1u;
    int rbase = __popc(s_head[w0] & (sh == 31 ? FULL : ((2u << sh) - 1u)));
    for (int w = 0; w < w0; ++w) rbase += __popc(s_head[w]);
    const bool first_head = (lane == 0) || (hv & 1u);
    bool next_head = true;
    if (lane < 31) {
      const int q = base + V;
      next_head = (s_head[q >> 5] >> (q & 31)) & 1u;
    }

    if (MODE == MIN_EDGE) {
      unsigned long long lead = KEY_INF, cur = KEY_INF;
      bool brk = false;
      int cr = rbase;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) {
          if (brk) {
            if (cur != KEY_INF) atomicMin(r + s_pi[cr], cur);
          } else {
            lead = cur;
          }
          brk = true;
          cur = KEY_INF;
          ++cr;
        }
        const unsigned long long cand = (pj[j] != s_pi[cr]) ? k[j] : KEY_INF;
        live += (cand != KEY_INF);
        cur = umin64(cur, cand);
      }
      // segmented inclusive min-scan of the trailing segments across lanes
      unsigned long long agg = cur;
      int f = (brk || first_head) ? 1 : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long oa = __shfl_up_sync(FULL, agg, d);
        const int of = __shfl_up_sync(FULL, f, d);
        if (lane >= d) {
          if (!f) agg = umin64(agg, oa);
          f |= of;
        }
      }
      unsigned long long prev = __shfl_up_sync(FULL, agg, 1);
      if (lane == 0) prev = KEY_INF;
      if (brk) {
        const unsigned long long v = first_head ? lead : umin64(prev, lead);
        if (v != KEY_INF) atomicMin(r + s_pi[rbase], v);
      }
      if (next_head && agg != KEY_INF) atomicMin(r + s_pi[cr], agg);
    } else if (MODE == COUNT) {
      unsigned long long lead = 0, cur = 0, tl = 0;
      bool brk = false;
      int cr = rbase;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) {
          if (brk) {
            if (cur) atomicAdd(rowcnt + k0 + cr, cur);
          } else {
            lead = cur;
          }
          brk = true;
          cur = 0;
          ++cr;
        }
        const int l = (sl + j < nnz) && (pj[j] != s_pi[cr]);
        cur += l;
        tl += l;
      }
      unsigned long long agg = cur;
      int f = (brk || first_head) ? 1 : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long oa = __shfl_up_sync(FULL, agg, d);
        const int of = __shfl_up_sync(FULL, f, d);
        if (lane >= d) {
          if (!f) agg += oa;
          f |= of;
        }
      }
      unsigned long long prev = __shfl_up_sync(FULL, agg, 1);
      if (lane == 0) prev = 0;
      if (brk) {
        const unsigned long long v = first_head ? lead : prev + lead;
        if (v) atomicAdd(rowcnt + k0 + rbase, v);
      }
      if (next_head && agg) atomicAdd(rowcnt + k0 + cr, agg);
      // live slots of this tile
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) tl += __shfl_xor_sync(FULL, tl, d);
      if (lane == 0) st->tilecnt[t] = (int64_t)tl;
    } else {  // SCATTER
      uint32_t lbits = 0;
      int cr = rbase;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) ++cr;
        if ((sl + j < nnz) && (pj[j] != s_pi[cr])) lbits |= 1u << j;
      }
      const int cnt = __popc(lbits);
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += o;
      }
      int64_t pos = st->tilecnt[t] + (incl - cnt);
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if ((lbits >> j) & 1u) {
          D.col[pos] = pj[j];
          D.key[pos] = k[j];
          ++pos;
        }
      }
    }
    __syncwarp();
  }

  if (MODE == MIN_EDGE) {
    // live slots this round, one atomic per block
    __shared__ unsigned long long blk_live;
    if (threadIdx.x == 0) blk_live = 0;
    __syncthreads();
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) live += __shfl_xor_sync(FULL, live, d);
    if (lane == 0 && live) atomicAdd(&blk_live, live);
    __syncthreads();
    if (threadIdx.x == 0 && blk_live) atomicAdd(&st->n_live, blk_live);
  }
  if (bad) st->status = MSF_ERR_CHECK;
}

// ---- compaction helpers ---------------------------------------------------------

__global__ void k_cmp_prep(DevState *st, int S) {
  const int64_t nr = st->nrows;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) st->rowcnt[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->scan_n[0] = (st->nnz + S - 1) / S;
    st->scan_n[1] = nr;
  }
}

__global__ void k_cmp_flags(DevState *st) {
  const int64_t nr = st->nrows;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride)
    st->rowflag[i] = st->rowcnt[i] > 0;
}

// New rows: row k keeps iff it has live slots; its vertex becomes its root.
__global__ void k_cmp_rows(DevState *st) {
  const CsrBuf B = st->buf[st->cur];
  const CsrBuf D = st->buf[st->cur == 1 ? 2 : 1];
  const int64_t nr = st->nrows, nnz_new = st->scan_tot[1], nr_new = st->scan_tot[2];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += stride) {
    const int64_t o = st->rowcnt[k];
    const int64_t on = (k + 1 < nr) ? st->rowcnt[k + 1] : nnz_new;
    if (on > o) {
      const int64_t kp = st->rowflag[k];
      D.rows[kp] = st->p[B.rows[k]];
      D.rp[kp] = o;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) D.rp[nr_new] = nnz_new;
}

__global__ void k_cmp_finish(DevState *st) {
  st->cur = st->cur == 1 ? 2 : 1;
  st->nrows = st->scan_tot[2];
  st->nnz = st->scan_tot[1];
  st->compactions += 1;
}

template <int V>
void launch_compact_v(DevState *st, cudaStream_t s, int grid) {
  constexpr int S = 32 * V;
  const int g2 = sm_count() * 4;
  k_cmp_prep<<<g2, 256, 0, s>>>(st, S);
  k_sweep<V, COUNT><<<grid, THREADS, 0, s>>>(st);
  k_cmp_flags<<<g2, 256, 0, s>>>(st);
  launch_scan_excl_ind(&st->tilecnt, &st->scan_n[0], &st->scan_tmp, &st->scan_tot[0], s);
  launch_scan_excl_ind(&st->rowcnt, &st->scan_n[1], &st->scan_tmp, &st->scan_tot[1], s);
  launch_scan_excl_ind(&st->rowflag, &st->scan_n[1], &st->scan_tmp, &st->scan_tot[2], s);
  k_cmp_rows<<<g2, 256, 0, s>>>(st);
  k_sweep<V, SCATTER><<<grid, THREADS, 0, s>>>(st);
  k_cmp_finish<<<1, 1, 0, s>>>(st);
  launch_tile_rows(st, -1, s);
}

}  // namespace

void launch_min_edge(DevState *st, int spl, int blocks_per_sm, cudaStream_t s) {
  const int grid = sm_count() * blocks_per_sm;
  switch (spl) {
    case 4: k_sweep<4, MIN_EDGE><<<grid, THREADS, 0, s>>>(st); break;
    case 16: k_sweep<16, MIN_EDGE><<<grid, THREADS, 0, s>>>(st); break;
    default: k_sweep<8, MIN_EDGE><<<grid, THREADS, 0, s>>>(st); break;
  }
}

void launch_compact(DevState *st, int spl, int blocks_per_sm, cudaStream_t s) {
  const int grid = sm_count() * blocks_per_sm;
  switch (spl) {
    case 4: launch_compact_v<4>(st, s, grid); break;
    case 16: launch_compact_v<16>(st, s, grid); break;
    default: launch_compact_v<8>(st, s, grid); break;
  }
}

}  // namespace msf

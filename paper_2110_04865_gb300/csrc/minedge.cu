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
// Lane l streams V columns and V keys (16-byte vector loads, evict-first).
// Bit 31 of a column word marks the first slot of a row, so each lane knows
// where its segments begin without reading the row offsets; a warp prefix
// sum of those marks numbers the rows that meet the tile, and the warp
// stages p of those rows in shared memory (one row-vertex read and one p
// gather per row).  Lanes gather p_j, build candidates, reduce their own
// segments, a segmented shuffle scan joins segments that cross lanes, and a
// single atomicMin per (row, tile) segment writes the projection r_{p_i}.
// Rows that span tiles get one atomicMin per tile.  With PF = 1 the next
// tile's columns and keys are loaded before the current tile is processed.
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
constexpr uint32_t COL_MASK = 0x7fffffffu;

// MIN_EDGE: the multilinear kernel of the forest; COUNT/SCATTER: compaction;
// CC_COND/CC_ANY: the neighbour-parent minimum of connected components
// (Sec. 2.4): p^h_i = min { p_j : p_j < p_i } (conditional) or
// min { p_j : p_j != p_i } (unconditional), projected onto the star root.
enum Mode { MIN_EDGE = 0, COUNT = 1, SCATTER = 2, CC_COND = 3, CC_ANY = 4 };

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

template <int V, bool KEYS>
__device__ __forceinline__ void load_tile(const CsrBuf &B, const int32_t *cw, int64_t sl, int32_t (&c)[V],
                                          uint64_t (&k)[V]) {
#pragma unroll
  for (int q = 0; q < V / 4; ++q) load_col4(cw + sl + 4 * q, c + 4 * q);
  if (KEYS) {
#pragma unroll
    for (int q = 0; q < V / 2; ++q) load_key2(B.key + sl + 2 * q, k + 2 * q);
  }
}

// PAIR = 1: the pairwise formulation's second pass -- the column words are
// replaced by the materialised parents p_j (with the same row marks), so the
// sweep reads (a_ij, p_j) pairs and gathers nothing.
template <int V, int MODE, int PF, int PAIR = 0>
__global__ void __launch_bounds__(THREADS, (V >= 16 ? 2 : 4)) k_sweep(DevState *st) {
  constexpr int S = 32 * V;
  constexpr int F = S / TB;
  constexpr bool KEYS = (MODE == MIN_EDGE || MODE == SCATTER);
  constexpr bool REDUCE = (MODE == MIN_EDGE || MODE == CC_COND || MODE == CC_ANY);
  __shared__ int32_t sm_pi[WARPS][S];  // p of the rows meeting the tile
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const CsrBuf B = st->buf[st->cur];
  const int32_t *cw = PAIR ? st->pjs : B.col;  // column words, or parents of the columns
  const int64_t nnz = st->nnz, nrows = st->nrows;
  const uint32_t nv = (uint32_t)st->n;
  const int32_t *__restrict__ p = st->p;
  const int32_t *__restrict__ prow = st->prow;
  const bool ident = REDUCE && st->first_round_identity != 0;
  unsigned long long *r = reinterpret_cast<unsigned long long *>(st->r);
  unsigned long long *rowcnt = reinterpret_cast<unsigned long long *>(st->rowcnt);
  const int64_t ntiles = (nnz + S - 1) / S;
  const int64_t tstride = (int64_t)gridDim.x * WARPS;
  int32_t *s_pi = sm_pi[wid];
  CsrBuf D;
  if (MODE == SCATTER) D = st->buf[st->cur == 1 ? 2 : 1];
  unsigned long long live = 0;
  bool bad = false;

  int64_t t = (int64_t)blockIdx.x * WARPS + wid;
  int32_t c[V];
  uint64_t k[V];
  int32_t k0 = 0;
  if (PF && t < ntiles) {
    load_tile<V, KEYS>(B, cw, t * S + (int64_t)lane * V, c, k);
    k0 = B.tile_row[t * F];
  }
  for (; t < ntiles; t += tstride) {
    const int64_t s0 = t * S;
    const int64_t sl = s0 + (int64_t)lane * V;
    // 1. the tile's slots (prefetched in the previous iteration when PF)
    if (!PF) {
      load_tile<V, KEYS>(B, cw, sl, c, k);
      k0 = B.tile_row[t * F];
    }
    int32_t cn[V];
    uint64_t kn[V];
    int32_t k0n = 0;
    const int64_t tn = t + tstride;
    if (PF && tn < ntiles) {
      load_tile<V, KEYS>(B, cw, tn * S + (int64_t)lane * V, cn, kn);
      k0n = B.tile_row[tn * F];
    }
    // 2. row starts in the lane's slots; number the rows meeting the tile
    uint32_t hv = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      hv |= ((uint32_t)c[j] >> 31) << j;
      c[j] &= (int32_t)COL_MASK;
    }
    const int cnt = __popc(hv);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += o;
    }
    const int head0 = __shfl_sync(FULL, (int)(hv & 1u), 0);
    const int total = __shfl_sync(FULL, incl, 31);
    int R = 1 + total - head0;                    // rows meeting the tile
    const int rbase = incl - cnt + (int)(hv & 1u) - head0;  // row of the lane's first slot
    const int nxt = __shfl_down_sync(FULL, (int)(hv & 1u), 1);
    const bool next_head = (lane == 31) || nxt;
    const bool first_head = (lane == 0) || (hv & 1u);
    if (k0 < 0 || (int64_t)k0 + R > nrows) {  // impossible for a consistent CSR
      bad = true;
      k0 = k0 < 0 ? 0 : (k0 >= nrows ? (int32_t)(nrows - 1) : k0);
      R = (int)((int64_t)k0 + R > nrows ? nrows - k0 : R);
    }
    // 3. stage p of those rows; gather p_j of the columns
    // p of the rows, from the per-row parent array written just before the
    // sweep (a row outside a star holds -1: its candidates are reduced but
    // never emitted, since the emission checks 0 <= p_i < n)
    for (int idx = lane; idx < R; idx += 32) s_pi[idx] = __ldg(prow + k0 + idx);
    int32_t pj[V];
#pragma unroll
    for (int j = 0; j < V; ++j) pj[j] = (PAIR || ident) ? c[j] : __ldg(p + c[j]);
    __syncwarp();
    int rb = rbase < 0 ? 0 : rbase;
    const int32_t pi0 = s_pi[rb];

    if (REDUCE) {
      unsigned long long lead = KEY_INF, cur = KEY_INF;
      bool brk = false;
      int32_t pi = pi0;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) {
          if (brk) {
            if (cur != KEY_INF && (uint32_t)pi < nv) atomicMin(r + pi, cur);
          } else {
            lead = cur;
          }
          brk = true;
          cur = KEY_INF;
          pi = s_pi[++rb];
        }
        unsigned long long cand;
        if (MODE == MIN_EDGE) cand = (pj[j] != pi) ? k[j] : KEY_INF;
        // (the padding slots after the last row carry no edge: their key is
        // the identity, but their column word is 0, so the parent candidates
        // of the connectivity sweeps must skip them explicitly)
        else if (MODE == CC_COND) cand = (sl + j < nnz && pj[j] < pi) ? (unsigned long long)pj[j] : KEY_INF;
        else cand = (sl + j < nnz && pj[j] != pi) ? (unsigned long long)pj[j] : KEY_INF;
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
        if (v != KEY_INF && (uint32_t)pi0 < nv) atomicMin(r + pi0, v);
      }
      if (next_head && agg != KEY_INF && (uint32_t)pi < nv) atomicMin(r + pi, agg);
    } else if (MODE == COUNT) {
      unsigned long long lead = 0, cur = 0, tl = 0;
      bool brk = false;
      int32_t pi = pi0;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) {
          if (brk) {
            if (cur) atomicAdd(rowcnt + k0 + rb, cur);
          } else {
            lead = cur;
          }
          brk = true;
          cur = 0;
          pi = s_pi[++rb];
        }
        const int l = (sl + j < nnz) && (pj[j] != pi);
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
        if (v) atomicAdd(rowcnt + k0 + (rbase < 0 ? 0 : rbase), v);
      }
      if (next_head && agg) atomicAdd(rowcnt + k0 + rb, agg);
      // live slots of this tile
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) tl += __shfl_xor_sync(FULL, tl, d);
      if (lane == 0) st->tilecnt[t] = (int64_t)tl;
    } else {  // SCATTER
      uint32_t lbits = 0;
      int32_t pi = pi0;
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) pi = s_pi[++rb];
        if ((sl + j < nnz) && (pj[j] != pi)) lbits |= 1u << j;
      }
      const int lc = __popc(lbits);
      int li = lc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, li, d);
        if (lane >= d) li += o;
      }
      int64_t pos = st->tilecnt[t] + (li - lc);
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if ((lbits >> j) & 1u) {
          D.col[pos] = pj[j];  // relabelled to the root; row marks are set afterwards
          D.key[pos] = k[j];
          ++pos;
        }
      }
    }
    __syncwarp();
    if (PF) {
#pragma unroll
      for (int j = 0; j < V; ++j) {
        c[j] = cn[j];
        if (KEYS) k[j] = kn[j];
      }
      k0 = k0n;
    }
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

// Per-row parents for the next sweep: prow[k] = p[rows[k]] (the identity in
// the first round), or -1 for a row outside a star when star flags are in
// use (original schedule, unconditional connectivity hooking).
__global__ void __launch_bounds__(256) k_prow(DevState *st, int use_star) {
  const CsrBuf B = st->buf[st->cur];
  const int64_t nr = st->nrows;
  const int32_t *p = st->p;
  const uint8_t *star = use_star ? st->star : nullptr;
  const bool ident = st->first_round_identity != 0;
  int32_t *out = st->prow;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += stride) {
    const int32_t v = B.rows[k];
    out[k] = (star && !star[v]) ? -1 : (ident ? v : p[v]);
  }
}

// Pairwise formulation, first pass g(a_ij, p_j) (Sec. 4.1): materialise the
// parent of every slot's column next to the slot (nnz extra writes), keeping
// the row marks.
__global__ void __launch_bounds__(256) k_pair_gather(DevState *st) {
  const CsrBuf B = st->buf[st->cur];
  const int32_t *p = st->p;
  int32_t *out = st->pjs;
  const bool ident = st->first_round_identity != 0;
  const int64_t padded = (st->nnz + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
  for (int64_t s4 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; s4 < padded; s4 += stride) {
    int32_t c[4];
    load_col4(B.col + s4, c);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int32_t head = c[j] & (int32_t)COL_HEAD;
      const int32_t col = c[j] & (int32_t)COL_MASK;
      c[j] = head | (ident ? col : __ldg(p + col));
    }
    *reinterpret_cast<int4 *>(out + s4) = make_int4(c[0], c[1], c[2], c[3]);
  }
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
  k_sweep<V, COUNT, 0><<<grid, THREADS, 0, s>>>(st);
  k_cmp_flags<<<g2, 256, 0, s>>>(st);
  launch_scan_excl_ind(&st->tilecnt, &st->scan_n[0], &st->scan_tmp, &st->scan_tot[0], s);
  launch_scan_excl_ind(&st->rowcnt, &st->scan_n[1], &st->scan_tmp, &st->scan_tot[1], s);
  launch_scan_excl_ind(&st->rowflag, &st->scan_n[1], &st->scan_tmp, &st->scan_tot[2], s);
  k_cmp_rows<<<g2, 256, 0, s>>>(st);
  k_sweep<V, SCATTER, 0><<<grid, THREADS, 0, s>>>(st);
  k_cmp_finish<<<1, 1, 0, s>>>(st);
  launch_tile_rows(st, -1, s);
}

}  // namespace

void launch_prow(DevState *st, int use_star, cudaStream_t s) {
  k_prow<<<sm_count() * 8, 256, 0, s>>>(st, use_star);
}

void launch_min_edge(DevState *st, int spl, int blocks_per_sm, int prefetch, cudaStream_t s, int pairwise) {
  const int grid = sm_count() * blocks_per_sm;
  if (pairwise) {
    k_pair_gather<<<sm_count() * 8, 256, 0, s>>>(st);
    switch (spl) {
      case 4: k_sweep<4, MIN_EDGE, 0, 1><<<grid, THREADS, 0, s>>>(st); break;
      case 16: k_sweep<16, MIN_EDGE, 0, 1><<<grid, THREADS, 0, s>>>(st); break;
      default: k_sweep<8, MIN_EDGE, 0, 1><<<grid, THREADS, 0, s>>>(st); break;
    }
    return;
  }
  if (prefetch) {
    switch (spl) {
      case 4: k_sweep<4, MIN_EDGE, 1><<<grid, THREADS, 0, s>>>(st); break;
      case 16: k_sweep<16, MIN_EDGE, 1><<<grid, THREADS, 0, s>>>(st); break;
      default: k_sweep<8, MIN_EDGE, 1><<<grid, THREADS, 0, s>>>(st); break;
    }
  } else {
    switch (spl) {
      case 4: k_sweep<4, MIN_EDGE, 0><<<grid, THREADS, 0, s>>>(st); break;
      case 16: k_sweep<16, MIN_EDGE, 0><<<grid, THREADS, 0, s>>>(st); break;
      default: k_sweep<8, MIN_EDGE, 0><<<grid, THREADS, 0, s>>>(st); break;
    }
  }
}

void launch_cc_sweep(DevState *st, bool conditional, cudaStream_t s) {
  const int grid = sm_count() * 4;
  k_prow<<<sm_count() * 8, 256, 0, s>>>(st, conditional ? 0 : 1);
  if (conditional) k_sweep<4, CC_COND, 0><<<grid, THREADS, 0, s>>>(st);
  else k_sweep<4, CC_ANY, 0><<<grid, THREADS, 0, s>>>(st);
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

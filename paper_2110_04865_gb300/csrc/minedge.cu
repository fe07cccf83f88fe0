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
constexpr int CT_BITS = 8;         // combining table of the projection: 256 roots per block
constexpr int CT = 1 << CT_BITS;
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t COL_MASK = 0x7fffffffu;

// MIN_EDGE: the multilinear kernel of the forest; COUNT/SCATTER: compaction;
// CC_COND/CC_ANY: the neighbour-parent minimum of connected components
// (Sec. 2.4): p^h_i = min { p_j : p_j < p_i } (conditional) or
// min { p_j : j's tree is not a star } (unconditional: a star hooks only
// onto a tree that does not move in this step, so no cycle forms),
// projected onto the star root.
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

// Block-wide combining table for the projection r_{p_i}: once parents
// repeat (after the first round), many segments of a block target the same
// root; their minima meet in shared memory and reach r with one atomic per
// root and block instead of one per segment (same-address global atomics
// serialise in L2: on R-MAT 20 the last round's sweep took 2.8 times the
// first one's).  Direct-mapped; a slot is claimed by the first root that
// hashes to it, other roots go to r directly.  init() and flush() are
// called by every thread of the block.
struct Combine {
  int32_t key[CT];
  unsigned long long val[CT];
  __device__ void init() {
    for (int i = threadIdx.x; i < CT; i += blockDim.x) {
      key[i] = -1;
      val[i] = KEY_INF;
    }
    __syncthreads();
  }
  __device__ __forceinline__ void emit(int32_t root, unsigned long long v, unsigned long long *r) {
    const int slot = (int)(((uint32_t)root * 0x9E3779B1u) >> (32 - CT_BITS));
    int kk = *reinterpret_cast<volatile int32_t *>(key + slot);
    if (kk == -1) {
      const int old = atomicCAS(key + slot, -1, root);
      kk = old == -1 ? root : old;
    }
    if (kk == root) atomicMin(val + slot, v);
    else atomicMin(r + root, v);
  }
  __device__ void flush(unsigned long long *r) {
    __syncthreads();
    for (int i = threadIdx.x; i < CT; i += blockDim.x)
      if (key[i] >= 0 && val[i] != KEY_INF) atomicMin(r + key[i], val[i]);
  }
};

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
// RELAB: the instantiation that runs the second round of a MIN_EDGE loop
// with relabelling on; the launcher starts both, and the one whose case it is
// not returns at once (the relabelling stores would otherwise cost the
// other rounds' kernel registers).
template <int V, int MODE, int PF, int PAIR = 0, bool RELAB = false>
__global__ void __launch_bounds__(THREADS, (V >= 16 ? 2 : 4)) k_sweep(DevState *st) {
  constexpr int S = 32 * V;
  constexpr int F = S / TB;
  constexpr bool KEYS = (MODE == MIN_EDGE || MODE == SCATTER);
  constexpr bool REDUCE = (MODE == MIN_EDGE || MODE == CC_COND || MODE == CC_ANY);
  // MIN_EDGE reads p of each slot's row straight from prow (consecutive
  // slots of a row load one address: L1 hits); the other modes stage the
  // parents of the rows meeting the tile in shared memory.  Less shared
  // memory leaves more of the SM's storage to L1 for the p_j gathers.
  constexpr bool DIRECT = (MODE == MIN_EDGE);
  __shared__ int32_t sm_pi[WARPS][DIRECT ? 1 : S];  // p of the rows meeting the tile
  __shared__ Combine comb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const CsrBuf B = st->buf[st->cur];
  const int32_t *cw = PAIR ? st->pjs : B.col;  // column words, or parents of the columns
  const int64_t nnz = st->nnz, nrows = st->nrows;
  const uint32_t nv = (uint32_t)st->n;
  const int32_t *__restrict__ p = st->p;
  const int32_t *__restrict__ prow = st->prow;
  const uint8_t *__restrict__ star = st->star;  // CC_ANY: star flags of the columns
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
  const bool combine = REDUCE && !ident && st->combine != 0;
  // the second round's sweep writes each slot's column as its current root
  // (p_j, with the row-start mark) into colr; from the third round on the
  // sweeps read colr, whose p_j gathers touch only the roots left after the
  // first round (k_round_end switches buf[0].col to it)
  const bool relab_round =
      MODE == MIN_EDGE && !PAIR && V % 4 == 0 && st->colr && st->round == 1 && st->cur == 0 && !ident;
  if (RELAB != relab_round) return;  // (uniform: before any barrier)
  int32_t *relab = RELAB ? st->colr : nullptr;
  if (combine) comb.init();
  auto emit = [&](int32_t root, unsigned long long v) {
    if (combine) comb.emit(root, v, r);
    else atomicMin(r + root, v);
  };

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
    if (!DIRECT)
      for (int idx = lane; idx < R; idx += 32) s_pi[idx] = __ldg(prow + k0 + idx);
    int32_t pj[V];
#pragma unroll
    for (int j = 0; j < V; ++j) pj[j] = (PAIR || ident) ? c[j] : __ldg(p + c[j]);
    const int32_t *prow_t = prow + k0;  // DIRECT: p of the tile's rows, read at each row start
    if (RELAB) {
#pragma unroll
      for (int q = 0; q < V / 4; ++q) {
        int4 o;
        o.x = pj[4 * q + 0] | (int32_t)(((hv >> (4 * q + 0)) & 1u) << 31);
        o.y = pj[4 * q + 1] | (int32_t)(((hv >> (4 * q + 1)) & 1u) << 31);
        o.z = pj[4 * q + 2] | (int32_t)(((hv >> (4 * q + 2)) & 1u) << 31);
        o.w = pj[4 * q + 3] | (int32_t)(((hv >> (4 * q + 3)) & 1u) << 31);
        __stcs(reinterpret_cast<int4 *>(relab + sl + 4 * q), o);
      }
    }
    uint32_t sj = 0;  // CC_ANY: bit j set when column j lies in a star
    if (MODE == CC_ANY) {
#pragma unroll
      for (int j = 0; j < V; ++j) sj |= (uint32_t)(__ldg(star + c[j]) != 0) << j;
    }
    __syncwarp();
    int rb = rbase < 0 ? 0 : rbase;
    const int32_t pi0 = DIRECT ? __ldg(prow_t + (rb < R ? rb : R - 1)) : s_pi[rb];

    if (REDUCE) {
      unsigned long long lead = KEY_INF, cur = KEY_INF;
      bool brk = false;
      int32_t pi = pi0;
      uint32_t lm = 0;  // live slots of the lane (p_i != p_j)
#pragma unroll
      for (int j = 0; j < V; ++j) {
        if (j > 0 && ((hv >> j) & 1u)) {
          if (brk) {
            if (cur != KEY_INF && (uint32_t)pi < nv) emit(pi, cur);
          } else {
            lead = cur;
          }
          brk = true;
          cur = KEY_INF;
          ++rb;
          pi = DIRECT ? __ldg(prow_t + (rb < R ? rb : R - 1)) : s_pi[rb];
        }
        if (MODE == MIN_EDGE) {
          const bool lv = pj[j] != pi;
          lm |= lv ? 1u << j : 0u;
          if (lv && k[j] < cur) cur = k[j];
        } else {
          // (the padding slots after the last row carry no edge: their key
          // is the identity, but their column word is 0, so the parent
          // candidates of the connectivity sweeps skip them explicitly)
          unsigned long long cand;
          if (MODE == CC_COND) cand = (sl + j < nnz && pj[j] < pi) ? (unsigned long long)pj[j] : KEY_INF;
          else cand = (sl + j < nnz && !((sj >> j) & 1u) && pj[j] != pi) ? (unsigned long long)pj[j] : KEY_INF;
          live += (cand != KEY_INF);
          cur = umin64(cur, cand);
        }
      }
      if (MODE == MIN_EDGE) {
        // padding slots after the last row are not counted as live
        const int64_t nvalid = nnz - sl;
        if (nvalid < V) lm &= nvalid <= 0 ? 0u : (1u << nvalid) - 1u;
        live += __popc(lm);
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
        if (v != KEY_INF && (uint32_t)pi0 < nv) emit(pi0, v);
      }
      if (next_head && agg != KEY_INF && (uint32_t)pi < nv) emit(pi, agg);
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

  if (combine) comb.flush(r);
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

// ---- pipelined min-edge sweep ----------------------------------------------------
//
// The same multilinear min-edge computation as k_sweep<V, MIN_EDGE>, with the
// memory traffic decoupled from the registers: every warp owns a ring of NS
// shared-memory stages and works two tiles ahead.  For tile i+2 one lane
// issues two bulk copies (cp.async.bulk, columns and keys) that complete on
// the stage's mbarrier; for tile i+1, whose columns have arrived, the lanes
// issue 4-byte cp.async gathers of p_j and of the parents of the rows that
// meet the tile; tile i is then reduced from shared memory.  Waits on an
// mbarrier are bounded: on a timeout the warp records MSF_ERR_CHECK, waits
// (bounded again) for its copies and stops.

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// true once the phase with the given parity has completed; false after
// `limit` unsuccessful polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit) {
  const uint32_t a = smem_u32(bar);
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr unsigned MBAR_POLLS = 1u << 20;  // well over any copy's latency

template <int V>
struct PipeStage {
  int32_t col[32 * V];   // column words (bulk copy)
  uint64_t key[32 * V];  // keys (bulk copy)
  int32_t pj[32 * V];    // p of the columns (gathered)
  int32_t pi[32 * V];    // p of the rows meeting the tile (gathered from prow)
};

template <int V, int NS, int W>
constexpr size_t pipe_smem() {
  return (size_t)W * NS * sizeof(PipeStage<V>) + (size_t)W * NS * 8;
}

template <int V, int NS, int W>
__global__ void __launch_bounds__(W * 32) k_sweep_pipe(DevState *st) {
  constexpr int S = 32 * V;
  constexpr int F = S / TB;
  static_assert(V % 4 == 0 && NS >= 3, "tile shape");
  extern __shared__ __align__(128) unsigned char pipe_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PipeStage<V> *stg = reinterpret_cast<PipeStage<V> *>(pipe_raw) + wid * NS;
  uint64_t *bar = reinterpret_cast<uint64_t *>(pipe_raw + (size_t)W * NS * sizeof(PipeStage<V>)) + wid * NS;

  const CsrBuf B = st->buf[st->cur];
  const int64_t nnz = st->nnz, nrows = st->nrows;
  const uint32_t nv = (uint32_t)st->n;
  const int32_t *__restrict__ p = st->p;
  const int32_t *__restrict__ prow = st->prow;
  const bool ident = st->first_round_identity != 0;
  unsigned long long *r = reinterpret_cast<unsigned long long *>(st->r);
  const int64_t ntiles = (nnz + S - 1) / S;
  const int64_t stride = (int64_t)gridDim.x * W;
  const int64_t t0 = (int64_t)blockIdx.x * W + wid;
  unsigned long long live = 0;
  bool bad = false, timeout = false;
  __shared__ Combine comb;
  const bool combine = !ident && st->combine != 0;
  if (combine) comb.init();
  auto emit = [&](int32_t root, unsigned long long v) {
    if (combine) comb.emit(root, v, r);
    else atomicMin(r + root, v);
  };
  uint32_t phase = 0;  // parity bit per stage
  int64_t issued = 0;  // tiles whose bulk copies were issued
  int64_t waited = 0;  // tiles whose bulk copies were waited for

  if (lane == 0) {
    for (int q = 0; q < NS; ++q) mbar_init(bar + q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // first rows of the warp's tiles, 32 tiles per register batch: lane l of
  // batch b holds tile_row of local tile 32 b + l; the next batch is loaded
  // a batch ahead
  auto k0_batch = [&](int64_t b) -> int32_t {
    const int64_t t = t0 + (32 * b + lane) * stride;
    return t < ntiles ? __ldg(B.tile_row + t * F) : 0;
  };
  int64_t kbat = 0;
  int32_t kcur = k0_batch(0), knext = k0_batch(1);

  // lane 0 starts the bulk copies of the warp's local tile i into stage i % NS
  auto issue = [&](int64_t i) {
    const int64_t t = t0 + i * stride;
    if (t >= ntiles) return;
    issued = i + 1;
    if (lane == 0) {
      const int q = (int)(i % NS);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar + q, (unsigned)(S * 12));
      bulk_g2s(stg[q].col, B.col + t * S, S * 4, bar + q);
      bulk_g2s(stg[q].key, B.key + t * S, S * 8, bar + q);
    }
  };
  // waits for tile i's columns and starts its gathers (one cp.async group,
  // possibly empty)
  auto gather = [&](int64_t i) {
    const int64_t t = t0 + i * stride;
    if (t < ntiles && !timeout) {
      const int q = (int)(i % NS);
      if (!__all_sync(FULL, mbar_wait(bar + q, (phase >> q) & 1u, MBAR_POLLS))) {
        timeout = true;
      } else {
        phase ^= 1u << q;
        ++waited;
        __syncwarp();
        int32_t c[V];
#pragma unroll
        for (int j = 0; j < V; j += 4) {
          const int4 x = *reinterpret_cast<const int4 *>(&stg[q].col[lane * V + j]);
          c[j] = x.x;
          c[j + 1] = x.y;
          c[j + 2] = x.z;
          c[j + 3] = x.w;
        }
        unsigned heads = 0;
#pragma unroll
        for (int j = 0; j < V; ++j) {
          heads += (uint32_t)c[j] >> 31;
          if (!ident) cp_async4(&stg[q].pj[lane * V + j], p + (c[j] & (int32_t)COL_MASK));
        }
        const unsigned total = __reduce_add_sync(FULL, heads);
        const int head0 = (int)((uint32_t)stg[q].col[0] >> 31);
        if (i / 32 != kbat) {
          kcur = knext;
          ++kbat;
          knext = k0_batch(kbat + 1);
        }
        int32_t k0 = __shfl_sync(FULL, kcur, (int)(i % 32));
        int R = 1 + (int)total - head0;
        if (k0 < 0 || (int64_t)k0 + R > nrows) {  // impossible for a consistent CSR
          bad = true;
          k0 = k0 < 0 ? 0 : (k0 >= nrows ? (int32_t)(nrows - 1) : k0);
          R = (int)((int64_t)k0 + R > nrows ? nrows - k0 : R);
        }
        for (int idx = lane; idx < R; idx += 32) cp_async4(&stg[q].pi[idx], prow + k0 + idx);
      }
    }
    cp_async_commit();
  };

  issue(0);
  issue(1);
  gather(0);
  for (int64_t i = 0; t0 + i * stride < ntiles && !timeout; ++i) {
    issue(i + 2);
    gather(i + 1);
    cp_async_wait<1>();  // tile i's gathers
    __syncwarp();
    if (timeout) break;
    const int q = (int)(i % NS);
    const PipeStage<V> &sg = stg[q];
    int32_t c[V], pj[V];
    uint64_t k[V];
#pragma unroll
    for (int j = 0; j < V; j += 4) {
      const int4 x = *reinterpret_cast<const int4 *>(&sg.col[lane * V + j]);
      c[j] = x.x;
      c[j + 1] = x.y;
      c[j + 2] = x.z;
      c[j + 3] = x.w;
      if (!ident) {
        const int4 y = *reinterpret_cast<const int4 *>(&sg.pj[lane * V + j]);
        pj[j] = y.x;
        pj[j + 1] = y.y;
        pj[j + 2] = y.z;
        pj[j + 3] = y.w;
      }
      const ulonglong2 k01 = *reinterpret_cast<const ulonglong2 *>(&sg.key[lane * V + j]);
      const ulonglong2 k23 = *reinterpret_cast<const ulonglong2 *>(&sg.key[lane * V + j + 2]);
      k[j] = k01.x;
      k[j + 1] = k01.y;
      k[j + 2] = k23.x;
      k[j + 3] = k23.y;
    }
    // row starts in the lane's slots; number of the lane's first row
    uint32_t hv = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      hv |= ((uint32_t)c[j] >> 31) << j;
      c[j] &= (int32_t)COL_MASK;
      if (ident) pj[j] = c[j];
    }
    const int cnt = __popc(hv);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += o;
    }
    const int head0 = __shfl_sync(FULL, (int)(hv & 1u), 0);
    const int rbase = incl - cnt + (int)(hv & 1u) - head0;
    const int nxt = __shfl_down_sync(FULL, (int)(hv & 1u), 1);
    const bool next_head = (lane == 31) || nxt;
    const bool first_head = (lane == 0) || (hv & 1u);
    int rb = rbase < 0 ? 0 : rbase;
    const int32_t pi0 = sg.pi[rb];
    unsigned long long lead = KEY_INF, cur = KEY_INF;
    bool brk = false;
    int32_t pi = pi0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if (j > 0 && ((hv >> j) & 1u)) {
        if (brk) {
          if (cur != KEY_INF && (uint32_t)pi < nv) emit(pi, cur);
        } else {
          lead = cur;
        }
        brk = true;
        cur = KEY_INF;
        pi = sg.pi[++rb];
      }
      const unsigned long long cand = (pj[j] != pi) ? k[j] : KEY_INF;
      live += (cand != KEY_INF);
      cur = umin64(cur, cand);
    }
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
      if (v != KEY_INF && (uint32_t)pi0 < nv) emit(pi0, v);
    }
    if (next_head && agg != KEY_INF && (uint32_t)pi < nv) emit(pi, agg);
    __syncwarp();  // stage q is refilled by issue(i + NS) at the earliest
  }
  cp_async_wait<0>();
  if (timeout) {
    // let the bulk copies still in flight land before the block exits
    for (int64_t i = waited; i < issued; ++i) {
      const int q = (int)(i % NS);
      mbar_wait(bar + q, (phase >> q) & 1u, MBAR_POLLS);
      phase ^= 1u << q;
    }
  }
  if (combine) comb.flush(r);
  __shared__ unsigned long long blk_live;
  if (threadIdx.x == 0) blk_live = 0;
  __syncthreads();
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) live += __shfl_xor_sync(FULL, live, d);
  if (lane == 0 && live) atomicAdd(&blk_live, live);
  __syncthreads();
  if (threadIdx.x == 0 && blk_live) atomicAdd(&st->n_live, blk_live);
  if (bad || timeout) st->status = MSF_ERR_CHECK;
}

// ---- register-pipelined min-edge sweep ---------------------------------------------
//
// The register-tile sweep with its dependent loads moved ahead: in the step
// that reduces tile i, a warp loads the columns and keys of tile i+2 and
// gathers p_j of tile i+1 (whose columns arrived during the previous step)
// and, by cp.async into a double-buffered shared array, the parents of the
// rows that meet tile i+1.  The first rows of the tiles come 32 tiles at a
// time, one per lane.

__device__ __forceinline__ void ld_tile(const int32_t *col, const uint64_t *key, int64_t sl, int V4,
                                        int32_t *c, uint64_t *k) {
  for (int q = 0; q < V4; ++q) {
    const int4 x = __ldcs(reinterpret_cast<const int4 *>(col + sl) + q);
    c[4 * q] = x.x;
    c[4 * q + 1] = x.y;
    c[4 * q + 2] = x.z;
    c[4 * q + 3] = x.w;
    const ulonglong2 a = __ldcs(reinterpret_cast<const ulonglong2 *>(key + sl) + 2 * q);
    const ulonglong2 b = __ldcs(reinterpret_cast<const ulonglong2 *>(key + sl) + 2 * q + 1);
    k[4 * q] = a.x;
    k[4 * q + 1] = a.y;
    k[4 * q + 2] = b.x;
    k[4 * q + 3] = b.y;
  }
}

template <int V>
__global__ void __launch_bounds__(THREADS, 3) k_sweep_deep(DevState *st) {
  constexpr int S = 32 * V;
  constexpr int F = S / TB;
  __shared__ int32_t sm_pi[WARPS][2][S];  // parents of the rows meeting tiles i and i+1
  __shared__ Combine comb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const CsrBuf B = st->buf[st->cur];
  const int64_t nnz = st->nnz, nrows = st->nrows;
  const uint32_t nv = (uint32_t)st->n;
  const int32_t *__restrict__ p = st->p;
  const int32_t *__restrict__ prow = st->prow;
  const bool ident = st->first_round_identity != 0;
  unsigned long long *r = reinterpret_cast<unsigned long long *>(st->r);
  const int64_t ntiles = (nnz + S - 1) / S;
  const int64_t stride = (int64_t)gridDim.x * WARPS;
  const int64_t t0 = (int64_t)blockIdx.x * WARPS + wid;
  unsigned long long live = 0;
  bool bad = false;
  const bool combine = !ident && st->combine != 0;
  if (combine) comb.init();
  auto emit = [&](int32_t root, unsigned long long v) {
    if (combine) comb.emit(root, v, r);
    else atomicMin(r + root, v);
  };

  auto k0_batch = [&](int64_t b) -> int32_t {
    const int64_t t = t0 + (32 * b + lane) * stride;
    return t < ntiles ? __ldg(B.tile_row + t * F) : 0;
  };
  int64_t kbat = 0;
  int32_t kcur = k0_batch(0), knext = k0_batch(1);
  auto tile_of = [&](int64_t i) { return t0 + i * stride; };

  int32_t c0[V], c1[V], c2[V], pj0[V], pj1[V];
  uint64_t k0v[V], k1v[V], k2v[V];
  // prologue: tiles 0 and 1 loaded, tile 0's gathers issued
  if (tile_of(0) < ntiles) ld_tile(B.col, B.key, tile_of(0) * S + (int64_t)lane * V, V / 4, c1, k1v);
  if (tile_of(1) < ntiles) ld_tile(B.col, B.key, tile_of(1) * S + (int64_t)lane * V, V / 4, c2, k2v);

  // gathers for local tile i held in (c1, k1v): p_j into pj1 (registers,
  // consumed a step later), row parents by cp.async into sm_pi[wid][i & 1]
  auto gather = [&](int64_t i) {
    if (tile_of(i) >= ntiles) return;
    unsigned heads = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      heads += (uint32_t)c1[j] >> 31;
      const int32_t cc = c1[j] & (int32_t)COL_MASK;
      pj1[j] = ident ? cc : __ldg(p + cc);
    }
    const unsigned total = __reduce_add_sync(FULL, heads);
    const int head0 = __shfl_sync(FULL, (int)((uint32_t)c1[0] >> 31), 0);
    if (i / 32 != kbat) {
      kcur = knext;
      ++kbat;
      knext = k0_batch(kbat + 1);
    }
    int32_t k0 = __shfl_sync(FULL, kcur, (int)(i % 32));
    int R = 1 + (int)total - head0;
    if (k0 < 0 || (int64_t)k0 + R > nrows) {  // impossible for a consistent CSR
      bad = true;
      k0 = k0 < 0 ? 0 : (k0 >= nrows ? (int32_t)(nrows - 1) : k0);
      R = (int)((int64_t)k0 + R > nrows ? nrows - k0 : R);
    }
    int32_t *dst = sm_pi[wid][i & 1];
    for (int idx = lane; idx < R; idx += 32) cp_async4(dst + idx, prow + k0 + idx);
  };

  // rotate: tile 0 becomes current, tile 1 is gathered
#pragma unroll
  for (int j = 0; j < V; ++j) {
    c0[j] = c1[j];
    k0v[j] = k1v[j];
    c1[j] = c2[j];
    k1v[j] = k2v[j];
  }
  {
    // gather tile 0 (now in c0): temporarily move it back into the gather slot
    int32_t tc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
      tc[j] = c1[j];
      c1[j] = c0[j];
    }
    gather(0);
#pragma unroll
    for (int j = 0; j < V; ++j) {
      c1[j] = tc[j];
      pj0[j] = pj1[j];
    }
  }
  cp_async_commit();

  for (int64_t i = 0; tile_of(i) < ntiles; ++i) {
    const int64_t t = tile_of(i);
    if (tile_of(i + 2) < ntiles) ld_tile(B.col, B.key, tile_of(i + 2) * S + (int64_t)lane * V, V / 4, c2, k2v);
    gather(i + 1);
    cp_async_commit();
    cp_async_wait<1>();  // row parents of tile i
    __syncwarp();
    const int32_t *s_pi = sm_pi[wid][i & 1];
    // reduce tile i (c0, k0v, pj0)
    int32_t c[V];
    uint32_t hv = 0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      hv |= ((uint32_t)c0[j] >> 31) << j;
      c[j] = c0[j] & (int32_t)COL_MASK;
    }
    (void)t;
    (void)c;
    const int cnt = __popc(hv);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += o;
    }
    const int head0 = __shfl_sync(FULL, (int)(hv & 1u), 0);
    const int rbase = incl - cnt + (int)(hv & 1u) - head0;
    const int nxt = __shfl_down_sync(FULL, (int)(hv & 1u), 1);
    const bool next_head = (lane == 31) || nxt;
    const bool first_head = (lane == 0) || (hv & 1u);
    int rb = rbase < 0 ? 0 : rbase;
    const int32_t pi0 = s_pi[rb];
    unsigned long long lead = KEY_INF, cur = KEY_INF;
    bool brk = false;
    int32_t pi = pi0;
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if (j > 0 && ((hv >> j) & 1u)) {
        if (brk) {
          if (cur != KEY_INF && (uint32_t)pi < nv) emit(pi, cur);
        } else {
          lead = cur;
        }
        brk = true;
        cur = KEY_INF;
        pi = s_pi[++rb];
      }
      const unsigned long long cand = (pj0[j] != pi) ? k0v[j] : KEY_INF;
      live += (cand != KEY_INF);
      cur = umin64(cur, cand);
    }
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
      if (v != KEY_INF && (uint32_t)pi0 < nv) emit(pi0, v);
    }
    if (next_head && agg != KEY_INF && (uint32_t)pi < nv) emit(pi, agg);
    __syncwarp();  // sm_pi[wid][i & 1] is refilled by gather(i + 2)
#pragma unroll
    for (int j = 0; j < V; ++j) {
      c0[j] = c1[j];
      k0v[j] = k1v[j];
      pj0[j] = pj1[j];
      c1[j] = c2[j];
      k1v[j] = k2v[j];
    }
  }
  cp_async_wait<0>();
  if (combine) comb.flush(r);
  __shared__ unsigned long long blk_live;
  if (threadIdx.x == 0) blk_live = 0;
  __syncthreads();
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) live += __shfl_xor_sync(FULL, live, d);
  if (lane == 0 && live) atomicAdd(&blk_live, live);
  __syncthreads();
  if (threadIdx.x == 0 && blk_live) atomicAdd(&st->n_live, blk_live);
  if (bad) st->status = MSF_ERR_CHECK;
}

// Per-row parents for the next sweep: prow[k] = p[rows[k]] (the identity in
// the first round), or -1 for a row outside a star when star flags are in
// use (original schedule, unconditional connectivity hooking).
__global__ void __launch_bounds__(256) k_prow(DevState *st, int use_star) {
  if (st->prow_valid) return;  // the last round's shortcut pass already wrote it
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

// The register sweeps need little shared memory (row parents and the
// combining table, about 11 KB per block at 8 slots per lane), and their p_j
// gathers hit L1 often (high-degree columns recur).  Left to itself the
// driver may give most of each SM's 256 KB of L1/shared storage to shared
// memory; asking for just the shared memory the resident blocks use leaves
// the rest to L1 (R-MAT 26 sweep: 10.0 -> 9.25 ms).  Set once per device and
// kernel.
// `done`: bit d set once the attribute is set on device d (one word per kernel).
template <class F>
void prefer_l1(F *fn, int blocks_per_sm, unsigned long long &done) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && ((done >> dev) & 1ull)) return;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  // room for as many blocks as the registers allow (the grid's blocks per SM
  // may change between calls; the attribute is set once)
  (void)blocks_per_sm;
  int blocks = a.numRegs > 0 ? 65536 / (a.numRegs * THREADS) : 8;
  if (blocks > 2048 / THREADS) blocks = 2048 / THREADS;
  if (blocks < 1) blocks = 1;
  int smem_max = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (smem_max <= 0) smem_max = 228 * 1024;
  const double need = (double)blocks * ((double)a.sharedSizeBytes + 1024.0);
  int pct = (int)(100.0 * need / (double)smem_max) + 2;
  if (pct > 100) pct = 100;
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  cudaGetLastError();
  if (dev < 64) done |= 1ull << dev;
}

template <int V, int MODE, int PF, int PAIR = 0, bool RELAB = false>
void launch_sweep_one(DevState *st, int grid, int blocks_per_sm, cudaStream_t s) {
  static unsigned long long done = 0;
  prefer_l1(k_sweep<V, MODE, PF, PAIR, RELAB>, blocks_per_sm, done);
  k_sweep<V, MODE, PF, PAIR, RELAB><<<grid, THREADS, 0, s>>>(st);
}

// The register sweep; a MIN_EDGE sweep also starts its relabelling
// instantiation (which returns at once except in the second round).
template <int V, int MODE, int PF, int PAIR = 0>
void launch_sweep(DevState *st, int grid, int blocks_per_sm, cudaStream_t s) {
  launch_sweep_one<V, MODE, PF, PAIR, false>(st, grid, blocks_per_sm, s);
  if (MODE == MIN_EDGE && !PAIR) launch_sweep_one<V, MODE, PF, PAIR, true>(st, grid, blocks_per_sm, s);
}

template <int V>
void launch_compact_v(DevState *st, cudaStream_t s, int grid) {
  constexpr int S = 32 * V;
  const int g2 = sm_count() * 4;
  k_cmp_prep<<<g2, 256, 0, s>>>(st, S);
  launch_sweep<V, COUNT, 0>(st, grid, grid / sm_count(), s);
  k_cmp_flags<<<g2, 256, 0, s>>>(st);
  launch_scan_excl_ind(&st->tilecnt, &st->scan_n[0], &st->scan_tmp, &st->scan_tot[0], s);
  launch_scan_excl_ind(&st->rowcnt, &st->scan_n[1], &st->scan_tmp, &st->scan_tot[1], s);
  launch_scan_excl_ind(&st->rowflag, &st->scan_n[1], &st->scan_tmp, &st->scan_tot[2], s);
  k_cmp_rows<<<g2, 256, 0, s>>>(st);
  launch_sweep<V, SCATTER, 0>(st, grid, grid / sm_count(), s);
  k_cmp_finish<<<1, 1, 0, s>>>(st);
  launch_tile_rows(st, -1, s);
}

}  // namespace

void launch_prow(DevState *st, int use_star, cudaStream_t s) {
  k_prow<<<sm_count() * 8, 256, 0, s>>>(st, use_star);
}

template <int V, int NS, int W>
void launch_pipe(DevState *st, int blocks_per_sm, cudaStream_t s) {
  constexpr size_t smem = pipe_smem<V, NS, W>();
  static unsigned long long attr_set = 0;  // devices on which the attribute is set
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !((attr_set >> dev) & 1ull)) {
    cudaFuncSetAttribute(k_sweep_pipe<V, NS, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev < 64) attr_set |= 1ull << dev;
  }
  k_sweep_pipe<V, NS, W><<<sm_count() * blocks_per_sm, W * 32, smem, s>>>(st);
}

void launch_min_edge(DevState *st, int spl, int blocks_per_sm, int prefetch, cudaStream_t s, int pairwise) {
  const int grid = sm_count() * blocks_per_sm;
  if (!pairwise && options().sweep == 2) {
    switch (spl) {
      case 4: k_sweep_deep<4><<<grid, THREADS, 0, s>>>(st); break;
      case 16: k_sweep_deep<16><<<grid, THREADS, 0, s>>>(st); break;
      default: k_sweep_deep<8><<<grid, THREADS, 0, s>>>(st); break;
    }
    return;
  }
  if (!pairwise && options().sweep == 1) {
    switch (spl) {
      case 4: launch_pipe<4, 3, 8>(st, blocks_per_sm, s); break;
      case 16: launch_pipe<16, 3, 2>(st, blocks_per_sm, s); break;
      default: launch_pipe<8, 3, 4>(st, blocks_per_sm, s); break;
    }
    return;
  }
  const int b = blocks_per_sm;
  if (pairwise) {
    k_pair_gather<<<sm_count() * 8, 256, 0, s>>>(st);
    switch (spl) {
      case 4: launch_sweep<4, MIN_EDGE, 0, 1>(st, grid, b, s); break;
      case 16: launch_sweep<16, MIN_EDGE, 0, 1>(st, grid, b, s); break;
      default: launch_sweep<8, MIN_EDGE, 0, 1>(st, grid, b, s); break;
    }
    return;
  }
  if (prefetch) {
    switch (spl) {
      case 4: launch_sweep<4, MIN_EDGE, 1>(st, grid, b, s); break;
      case 16: launch_sweep<16, MIN_EDGE, 1>(st, grid, b, s); break;
      default: launch_sweep<8, MIN_EDGE, 1>(st, grid, b, s); break;
    }
  } else {
    switch (spl) {
      case 4: launch_sweep<4, MIN_EDGE, 0>(st, grid, b, s); break;
      case 16: launch_sweep<16, MIN_EDGE, 0>(st, grid, b, s); break;
      default: launch_sweep<8, MIN_EDGE, 0>(st, grid, b, s); break;
    }
  }
}

void launch_cc_sweep(DevState *st, bool conditional, cudaStream_t s) {
  const int grid = sm_count() * 4;
  k_prow<<<sm_count() * 8, 256, 0, s>>>(st, conditional ? 0 : 1);
  if (conditional) launch_sweep<4, CC_COND, 0>(st, grid, 4, s);
  else launch_sweep<4, CC_ANY, 0>(st, grid, 4, s);
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

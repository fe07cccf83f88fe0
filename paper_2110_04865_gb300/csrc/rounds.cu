// Per-round vertex kernels of Algorithm 2 and the end-of-run kernels.
//
//   hook       (Algorithm 2, hooking)        p_i <- r_i^parent for star roots with r_i
//   tie break  (Algorithm 2, tie breaking)   2-cycles: the smaller root keeps itself
//   shortcut   (Sec. 4.2, Algorithm 3)      complete shortcutting over the roots
//                                           whose parent changed, then one gather
//   round end  (Algorithm 2, loop test)      stop after a round without hooks
//   labels                                   smallest vertex id per component
//   sums       (Algorithm 2, weight update) exact forest weight per graph
//   backward                                 d(total)/d(w_e) = [e in forest]
// Every loop that waits on a condition is bounded: the round loop by
// round_limit, pointer jumping by jump_limit; exceeding either sets an error
// status that the host reads after the graph.
#include <cuda/atomic>

#include <mutex>
#include <string>

#include "internal.cuh"

namespace msf {

namespace {

constexpr int BT = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int64_t tid64() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t stride64() { return (int64_t)gridDim.x * blockDim.x; }

// The per-vertex passes over long lists (hooking, shortcutting, jumping)
// take UNR list entries per thread and step, each dependent load issued for
// all of them before the next: a grid-stride loop that finishes one entry
// before the next keeps one chain of dependent loads per thread in flight,
// which leaves these passes latency-bound on graphs with tens of millions
// of vertices.
constexpr int UNR = 4;

__device__ __forceinline__ int ld_relaxed(int *a) {
  return cuda::atomic_ref<int, cuda::thread_scope_device>(*a).load(cuda::memory_order_relaxed);
}
__device__ __forceinline__ void st_relaxed(int *a, int v) {
  cuda::atomic_ref<int, cuda::thread_scope_device>(*a).store(v, cuda::memory_order_relaxed);
}

__device__ __forceinline__ int32_t bsearch_off(const int64_t *off, int32_t G, int64_t x) {
  int32_t lo = 0, hi = G;  // off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_load_state(DevState *slot, DevState v) { *slot = v; }

// Adds the block's sum of `v` to *ctr with one atomic (a per-warp atomic on
// one counter serialises when a large graph launches ten thousand warps).
// Every thread of the block calls it.
__device__ __forceinline__ void block_add(unsigned long long *ctr, unsigned v) {
  __shared__ unsigned part[BT / 32];
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
#pragma unroll
    for (int w = 0; w < BT / 32; ++w) t += part[w];
    if (t) atomicAdd(ctr, (unsigned long long)t);
  }
}

__global__ void __launch_bounds__(BT) k_init(DevState *st) {
  const int64_t n = st->n, m = st->m;
  int32_t *p = st->p;
  uint64_t *r = st->r;
  for (int64_t v = tid64(); v < n; v += stride64()) {
    p[v] = (int32_t)v;
    r[v] = KEY_INF;
  }
  if (st->mask && st->mbits) {
    // the forest's bitmap (the mask itself is written whole at the end)
    uint4 *q = reinterpret_cast<uint4 *>(st->mbits);
    const int64_t nq = ((m + 31) / 32 + 2) / 4;
    for (int64_t i = tid64(); i < nq; i += stride64()) q[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t i = (nq << 2) + tid64(); i < (m + 31) / 32 + 2; i += stride64()) st->mbits[i] = 0u;
  } else if (st->mask) {
    // 16-byte stores between the unaligned head and tail of the caller's
    // byte array
    uint8_t *mask = st->mask;
    const int64_t head = (int64_t)((16 - (reinterpret_cast<uintptr_t>(mask) & 15)) & 15);
    const int64_t h = head < m ? head : m;
    const int64_t nq = (m - h) >> 4;
    for (int64_t e = tid64(); e < h; e += stride64()) mask[e] = 0;
    uint4 *q = reinterpret_cast<uint4 *>(mask + h);
    for (int64_t i = tid64(); i < nq; i += stride64()) q[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t e = h + (nq << 4) + tid64(); e < m; e += stride64()) mask[e] = 0;
  }
  const int64_t nb = (int64_t)st->G * 256;
  for (int64_t i = tid64(); i < nb; i += stride64()) st->bins[i] = 0;
}

// The vertices that may hook this round: every vertex under the original
// schedule (whose trees need not be stars), else the current roots among
// the non-isolated vertices, kept as a list that shrinks every round (the
// rows of the CSR at first; a root that did not hook stays in the list).
__device__ __forceinline__ int64_t hook_count(const DevState *st) {
  return st->rl_all ? st->n : (int64_t)st->rl_n;
}

// Algorithm 2, hooking (targets only): a root i with a minimum outgoing edge
// e = id(r_i) hooks onto the parent of e's endpoint outside i's star, read
// before any root moves; tgt holds the parent after hooking of every listed
// vertex, so tie breaking can read p_{p_i} from it.
__global__ void __launch_bounds__(BT) k_hook(DevState *st) {
  const int64_t cnt = hook_count(st);
  const int32_t *rl = st->rl_all ? nullptr : st->rl;
  const uint64_t *r = st->r;
  const int2 *ends = st->ends;
  const int32_t *p = st->p;
  int32_t *tgt = st->tgt;
  // first round: p is the identity, so no parent needs a gather
  const bool ident = st->first_round_identity != 0;
  // the row parents are stale from here until a shortcut pass rewrites them
  if (blockIdx.x == 0 && threadIdx.x == 0) st->prow_valid = 0;
  bool bad = false;
  unsigned active = 0;  // trees with an outgoing edge this round
  const int64_t stride = stride64();
  for (int64_t t0 = tid64(); t0 < cnt; t0 += UNR * stride) {
    int32_t iv[UNR], pu[UNR], pv[UNR];
    uint64_t rv[UNR];
    int2 uv[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t t = t0 + j * stride;
      iv[j] = t < cnt ? (rl ? rl[t] : (int32_t)t) : -1;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) rv[j] = iv[j] >= 0 ? r[iv[j]] : KEY_INF;
#pragma unroll
    for (int j = 0; j < UNR; ++j) uv[j] = rv[j] != KEY_INF ? ends[(uint32_t)rv[j]] : make_int2(iv[j], iv[j]);
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      if (iv[j] < 0) continue;
      if (rv[j] == KEY_INF) {
        // no hook: the parent stays (a listed vertex is a root)
        pu[j] = pv[j] = (ident || rl) ? iv[j] : p[iv[j]];
      } else {
        pu[j] = ident ? uv[j].x : p[uv[j].x];
        pv[j] = ident ? uv[j].y : p[uv[j].y];
      }
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      if (iv[j] < 0) continue;
      const int32_t i = iv[j];
      if (rv[j] == KEY_INF) {
        tgt[i] = pu[j];
        continue;
      }
      ++active;
      if (pu[j] != i && pv[j] != i) bad = true;
      tgt[i] = (pu[j] == i) ? pv[j] : pu[j];
    }
  }
  block_add(&st->n_active, active);
  if (bad) st->status = MSF_ERR_CHECK;
}

// Algorithm 2, tie breaking and weight update: t_i = (i < p_i and p_{p_i} = i)
// breaks each 2-cycle in favour of the smaller root; every other hooking
// root takes its parent, adds its edge to the forest and is appended to the
// changed list of Algorithm 3.  Roots that stay roots form the next round's
// list.
// Appends take their places with one atomic per block and chunk of
// TB_ITEMS * BT listed vertices (per-warp atomics on the two counters
// serialise on large graphs: half a million warps in the first round of the
// 256^3 grid); short lists use one vertex per thread and chunk, so that
// they still spread over many blocks.
template <int TB_ITEMS>
__device__ __forceinline__ void tiebreak_body(DevState *st, int64_t cnt) {
  const int32_t *rl = st->rl_all ? nullptr : st->rl;
  int32_t *rn = st->rl_next;
  uint64_t *r = st->r;
  const int32_t *tgt = st->tgt;
  int32_t *p = st->p;
  const unsigned long long msf_base = st->n_msf;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  __shared__ unsigned s_h[BT / 32], s_s[BT / 32];
  __shared__ unsigned long long s_hbase, s_sbase;
  const int64_t chunk = (int64_t)BT * TB_ITEMS;
  for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < cnt; c0 += (int64_t)gridDim.x * chunk) {
    bool hooks[TB_ITEMS], stays[TB_ITEMS];
    int32_t iv[TB_ITEMS], jv[TB_ITEMS];
    uint64_t rv[TB_ITEMS];
    // each dependent load for all items before the next (the resets of r
    // follow with the writes)
#pragma unroll
    for (int k = 0; k < TB_ITEMS; ++k) {
      const int64_t t = c0 + (int64_t)k * BT + threadIdx.x;
      iv[k] = t < cnt ? (rl ? rl[t] : (int32_t)t) : -1;
    }
#pragma unroll
    for (int k = 0; k < TB_ITEMS; ++k) rv[k] = iv[k] >= 0 ? r[iv[k]] : KEY_INF;
#pragma unroll
    for (int k = 0; k < TB_ITEMS; ++k) jv[k] = rv[k] != KEY_INF ? tgt[iv[k]] : 0;
#pragma unroll
    for (int k = 0; k < TB_ITEMS; ++k) {
      const int32_t back = rv[k] != KEY_INF ? tgt[jv[k]] : -1;  // p_{p_i}
      hooks[k] = rv[k] != KEY_INF && !((back == iv[k]) && (iv[k] < jv[k]));
      stays[k] = iv[k] >= 0 && !hooks[k];
    }
    unsigned bh[TB_ITEMS], bs[TB_ITEMS], wh = 0, ws = 0;
#pragma unroll
    for (int k = 0; k < TB_ITEMS; ++k) {
      bh[k] = __ballot_sync(FULL, hooks[k]);
      bs[k] = __ballot_sync(FULL, stays[k]);
      wh += __popc(bh[k]);
      ws += __popc(bs[k]);
    }
    if (lane == 0) {
      s_h[wid] = wh;
      s_s[wid] = ws;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned th = 0, ts = 0;
      for (int w = 0; w < BT / 32; ++w) {
        const unsigned a = s_h[w], c = s_s[w];
        s_h[w] = th;
        s_s[w] = ts;
        th += a;
        ts += c;
      }
      s_hbase = th ? atomicAdd(&st->n_hooks, (unsigned long long)th) : 0ull;
      s_sbase = (rl && ts) ? atomicAdd(&st->rl_next_n, (unsigned long long)ts) : 0ull;
    }
    __syncthreads();
    unsigned long long hb = s_hbase + s_h[wid], sb = s_sbase + s_s[wid];
#pragma unroll
    for (int k = 0; k < TB_ITEMS; ++k) {
      if (rv[k] != KEY_INF) r[iv[k]] = KEY_INF;  // identity for the next round
      if (hooks[k]) {
        const unsigned long long slot = hb + __popc(bh[k] & below);
        p[iv[k]] = jv[k];
        st->changed[slot] = iv[k];
        st->msf_keys[msf_base + slot] = rv[k];  // the mask is written from these at the end
      }
      hb += __popc(bh[k]);
      if (rl && stays[k]) rn[sb + __popc(bs[k] & below)] = iv[k];
      sb += __popc(bs[k]);
    }
    __syncthreads();  // s_h, s_s are rewritten by the next chunk
  }
}

__global__ void __launch_bounds__(BT) k_tiebreak(DevState *st) {
  const int64_t cnt = hook_count(st);
  if (cnt >= ((int64_t)1 << 20)) tiebreak_body<4>(st, cnt);
  else tiebreak_body<1>(st, cnt);
}

__global__ void k_jump_init(DevState *st, cudaGraphConditionalHandle h) {
  st->n_changed = st->n_hooks;
  st->jumps = 0;
  st->jump_dirty = 0;
  st->ticket = 0;
  const unsigned v = st->n_hooks > 0 ? 1u : 0u;
  st->ctl_jump = (int32_t)v;
  if (st->use_graph) cudaGraphSetConditional(h, v);
}

// Algorithm 3 on one device: every root in `changed` follows its parent
// chain towards the final root (the chase of the changed map), at most
// JUMP_HOPS hops per pass, and stores the farthest ancestor it reached.  In
// place: values only move up the hook tree, so reading a parent that another
// thread is updating still yields an ancestor.  A root whose chain did not
// end within the pass marks the pass dirty (another pass follows).
constexpr int JUMP_HOPS = 16;
__global__ void __launch_bounds__(BT) k_jump(DevState *st) {
  const unsigned long long nc = st->n_changed;
  int32_t *p = st->p;
  const int32_t *ch = st->changed;
  unsigned cnt = 0;
  const int64_t stride = stride64();
  for (int64_t t0 = tid64(); t0 < (int64_t)nc; t0 += UNR * stride) {
    // UNR chains followed side by side, one hop of each per step
    int v[UNR], x0[UNR], x[UNR];
    bool live[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t t = t0 + j * stride;
      v[j] = t < (int64_t)nc ? ch[t] : -1;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      x0[j] = v[j] >= 0 ? ld_relaxed(p + v[j]) : 0;
      x[j] = x0[j];
      live[j] = v[j] >= 0;
    }
#pragma unroll 1
    for (int h = 0; h < JUMP_HOPS; ++h) {
      bool any = false;
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        if (!live[j]) continue;
        const int y = ld_relaxed(p + x[j]);
        if (y == x[j]) live[j] = false;
        else x[j] = y;
        any |= live[j];
      }
      if (!any) break;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      if (v[j] < 0) continue;
      if (x[j] != x0[j]) st_relaxed(p + v[j], x[j]);
      cnt += live[j];  // chain not ended within the pass
    }
  }
  block_add(&st->jump_dirty, cnt);
}

// Another jumping step while some parent moved; bounded by jump_limit.
__global__ void k_jump_end(DevState *st, cudaGraphConditionalHandle h) {
  const unsigned long long dirty = st->jump_dirty;
  st->jump_dirty = 0;
  st->jumps += 1;
  st->jumps_total += 1;
  bool more = dirty > 0;
  if (more && st->jumps >= st->jump_limit) {
    st->status = MSF_ERR_SHORTCUT_LIMIT;
    more = false;
  }
  st->ctl_jump = more ? 1 : 0;
  if (st->use_graph) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// After the changed roots point at final roots, every vertex takes its
// grandparent: p_v was a root at the start of the round.
// Isolated vertices are roots throughout, so only the CSR's rows (the
// non-isolated vertices) are visited when they are known.
// While the edge list is the CSR as built (no compaction yet), the row
// parents of the next sweep are these final parents: the pass writes them
// too, and the next round's k_prow has nothing to do.
__global__ void __launch_bounds__(BT) k_shortcut_all(DevState *st) {
  if (st->n_changed == 0) return;
  const int32_t *rows = st->rl_all ? nullptr : st->buf[0].rows;
  const int64_t cnt = rows ? st->nrows0 : st->n;
  const bool rowp = rows && st->cur == 0;
  int32_t *prow = st->prow;
  int32_t *p = st->p;
  // (reading ahead of this thread's own writes is safe: a vertex's parent
  // is read only by the thread that owns the vertex, and the grandparents
  // read are roots, which this pass never writes)
  const int64_t stride = stride64();
  for (int64_t t0 = tid64(); t0 < cnt; t0 += UNR * stride) {
    int32_t v[UNR], x[UNR], y[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t t = t0 + j * stride;
      v[j] = t < cnt ? (rows ? rows[t] : (int32_t)t) : -1;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) x[j] = v[j] >= 0 ? p[v[j]] : 0;
#pragma unroll
    for (int j = 0; j < UNR; ++j) y[j] = v[j] >= 0 ? p[x[j]] : 0;
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      if (v[j] < 0) continue;
      if (y[j] != x[j]) p[v[j]] = y[j];
      if (rowp) prow[t0 + j * stride] = y[j];
    }
  }
  if (rowp && blockIdx.x == 0 && threadIdx.x == 0) st->prow_valid = 1;
}

__global__ void k_compact_decide(DevState *st, cudaGraphConditionalHandle h) {
  const int dst = st->cur == 1 ? 2 : 1;
  const unsigned long long live = st->n_live;
  const bool go = st->tau > 0.f && live > 0 && st->status == 0 &&
                  (double)live < (double)st->tau * (double)st->nnz &&
                  (int64_t)live <= st->buf[dst].cap_slots && st->nrows <= st->buf[dst].cap_rows;
  st->ctl_compact = go ? 1 : 0;
  if (st->use_graph) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Algorithm 2, loop test: continue while some star hooked.
__global__ void k_round_end(DevState *st, cudaGraphConditionalHandle h) {
  const unsigned long long hooks = st->n_hooks;
  // the second round's sweep wrote the relabelled columns: the later sweeps
  // (and a compaction) read them (after a compaction of the first round the
  // built CSR is no longer swept and nothing was written)
  if (st->colr && st->round == 1 && st->cur == 0) st->buf[0].col = st->colr;
  st->round += 1;
  st->n_msf += hooks;
  st->first_round_identity = 0;
  // the original schedule also continues while a shortcut step moved p
  bool more = (hooks > 0 || st->n_short > 0) && st->status == 0;
  // Early stop (complete shortcutting only): the trees that had an outgoing
  // edge this round merged into n_active - hooks trees.  If at most one is
  // left it has no outgoing edge (any such edge would lead to another tree
  // that had one too), so the round that would only confirm it is skipped.
  if (st->early_stop && st->shortcut_mode != MSF_SHORTCUT_ORIGINAL && hooks > 0 &&
      st->n_active <= hooks + 1ull)
    more = false;
  // Roots the next sweep can emit to: the trees with an outgoing edge merged
  // into n_active - hooks (connectivity does not count them: 0).  With far
  // fewer roots than rows, segments repeat their targets and the sweep
  // combines them per block.
  const unsigned long long left = st->n_active > hooks ? st->n_active - hooks : 0ull;
  st->combine = (double)left * 4.0 < (double)st->nrows ? 1 : 0;
  st->n_short = 0;
  st->n_active = 0;
  if (more && st->round >= st->round_limit) {
    st->status = MSF_ERR_ROUND_LIMIT;
    more = false;
  }
  st->n_hooks = 0;
  st->n_changed = 0;
  st->n_live = 0;
  // the roots that did not hook are the next round's list
  if (!st->rl_all) {
    st->rl = st->rl_next;
    st->rl_n = st->rl_next_n;
    st->rl_next = st->rl_next == st->rl_buf[0] ? st->rl_buf[1] : st->rl_buf[0];
    st->rl_next_n = 0;
  }
  st->ctl_round = more ? 1 : 0;
  if (st->use_graph) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---- star detection and the other shortcut schedules -------------------------
// Starcheck (Sec. 2.3): s_i = (p_i = p_{p_i}); a vertex whose parent is not a
// root clears its own flag and its grandparent's; then s_i <- s_{p_i}.
__global__ void __launch_bounds__(BT) k_star_init(DevState *st) {
  const int64_t n = st->n;
  for (int64_t v = tid64(); v < n; v += stride64()) st->star[v] = 1;
}

__global__ void __launch_bounds__(BT) k_star_mark(DevState *st) {
  const int64_t n = st->n;
  const int32_t *p = st->p;
  uint8_t *s = st->star;
  for (int64_t v = tid64(); v < n; v += stride64()) {
    const int32_t x = p[v], y = p[x];
    if (x != y) {
      s[v] = 0;
      s[y] = 0;
    }
  }
}

// Vertices still flagged take their parent's flag; the parent is then a
// root whose flag no thread changes in this kernel.
__global__ void __launch_bounds__(BT) k_star_pull(DevState *st) {
  const int64_t n = st->n;
  const int32_t *p = st->p;
  uint8_t *s = st->star;
  for (int64_t v = tid64(); v < n; v += stride64())
    if (s[v]) s[v] = s[p[v]];
}

// One shortcut step of the original schedule (Algorithm 1): every vertex
// outside a star takes its grandparent, all at once (into tgt, then copied).
__global__ void __launch_bounds__(BT) k_short_step(DevState *st) {
  const int64_t n = st->n;
  const int32_t *p = st->p;
  const uint8_t *s = st->star;
  int32_t *out = st->tgt;
  unsigned cnt = 0;
  for (int64_t v = tid64(); v < n; v += stride64()) {
    const int32_t x = p[v];
    const int32_t y = s[v] ? x : p[x];
    out[v] = y;
    cnt += (y != x);
  }
  block_add(&st->n_short, cnt);
}

__global__ void __launch_bounds__(BT) k_copy_parent(DevState *st) {
  const int64_t n = st->n;
  for (int64_t v = tid64(); v < n; v += stride64()) st->p[v] = st->tgt[v];
}

// Complete shortcutting by full passes (every vertex takes its grandparent,
// in place, until no parent moves): the one-device analogue of querying the
// parent vector in every sub-iteration.
__global__ void __launch_bounds__(BT) k_short_full(DevState *st) {
  const int64_t n = st->n;
  int32_t *p = st->p;
  unsigned cnt = 0;
  for (int64_t v = tid64(); v < n; v += stride64()) {
    const int x = ld_relaxed(p + v);
    const int y = ld_relaxed(p + x);
    if (x != y) {
      st_relaxed(p + v, y);
      ++cnt;
    }
  }
  block_add(&st->jump_dirty, cnt);
}

// Optimized shortcutting (Sec. 7.1): the changed-root chase when few roots
// changed, full passes otherwise.
__global__ void k_os_decide(DevState *st, cudaGraphConditionalHandle h) {
  const bool csp = (int64_t)st->n_hooks <= st->os_threshold;
  st->ctl_compact = csp ? 1 : 0;
  if (st->use_graph) cudaGraphSetConditional(h, csp ? 1u : 0u);
}

// ---- connected components (Sec. 2.4) -------------------------------------------
// A root with a candidate parent from the neighbour-parent sweep takes it:
// conditional candidates are smaller ids, unconditional ones lie in trees
// that are not stars (their roots do not move), so no cycle forms.
__global__ void __launch_bounds__(BT) k_cc_hook(DevState *st) {
  const int64_t n = st->n;
  uint64_t *r = st->r;
  int32_t *p = st->p;
  // parents have moved: the next sweep must gather them
  if (blockIdx.x == 0 && threadIdx.x == 0) st->first_round_identity = 0;
  unsigned cnt = 0;
  for (int64_t i = tid64(); i < n; i += stride64()) {
    const uint64_t ri = r[i];
    if (ri == KEY_INF) continue;
    r[i] = KEY_INF;
    p[i] = (int32_t)ri;
    ++cnt;
  }
  block_add(&st->n_hooks, cnt);
}

// ---- labels: the smallest vertex id of each tree ---------------------------
__global__ void __launch_bounds__(BT) k_label_init(DevState *st) {
  if (!st->labels) return;
  const int64_t n = st->n;
  for (int64_t v = tid64(); v < n; v += stride64()) st->tgt[v] = 0x7fffffff;
}

// Lanes of a warp that share a root offer their smallest id once (see below),
// so a root with many vertices (a giant component) takes about one atomic
// per warp instead of one per vertex.
__global__ void __launch_bounds__(BT) k_label_min(DevState *st) {
  if (!st->labels) return;
  const int64_t n = st->n;
  const int32_t *p = st->p;
  int32_t *lab = st->tgt;
  const int lane = threadIdx.x & 31;
  // the last root this lane offered a minimum for, and that minimum: a
  // large component's later vertices (higher ids) then need neither the
  // read nor the atomic on its root's word
  int32_t last_root = -1, last_min = 0x7fffffff;
  const int64_t stride = stride64();
  // UNR warp-wide groups per step, their parents loaded together; ids still
  // grow along a lane's groups
  for (int64_t b0 = tid64() - lane; b0 < n; b0 += UNR * stride) {
    int32_t roots[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t v = b0 + j * stride + lane;
      roots[j] = v < n ? p[v] : -1;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t i0 = b0 + j * stride;  // the same for every lane of the warp
      if (i0 >= n) break;
      const int64_t v = i0 + lane;
      const int32_t root = roots[j];
      // the lanes that share lane 0's root (a whole warp inside a large
      // component, or a large component's members among isolated vertices)
      // offer their smallest id once, from lane 0; every other lane offers its
      // own id (grouping all lanes by root with __match_any_sync costs more
      // than the atomics it saves on graphs with many isolated vertices)
      const int32_t root0 = __shfl_sync(FULL, root, 0);
      const unsigned m0 = __ballot_sync(FULL, root == root0);
      int32_t mn = (int32_t)v;
      if (root == root0) mn = m0 == FULL ? (int32_t)i0 : __reduce_min_sync(m0, (int32_t)v);
      if (v < n && (root != root0 || lane == 0) && !(root == last_root && mn >= last_min)) {
        // the read skips most atomics on a large component's root: ids
        // arrive roughly in increasing order, so its minimum is usually
        // known already
        if (mn < ld_relaxed(lab + root)) atomicMin(lab + root, mn);
        last_root = root;
        last_min = mn;
      }
    }
  }
}

__global__ void __launch_bounds__(BT) k_label_write(DevState *st) {
  if (!st->labels) return;
  const int64_t n = st->n;
  const int32_t G = st->G;
  const int32_t *p = st->p;
  const int32_t *lab = st->tgt;
  const int64_t stride = stride64();
  for (int64_t v0 = tid64(); v0 < n; v0 += UNR * stride) {
    int32_t r[UNR], l[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) r[j] = v0 + j * stride < n ? p[v0 + j * stride] : 0;
#pragma unroll
    for (int j = 0; j < UNR; ++j) l[j] = v0 + j * stride < n ? lab[r[j]] : 0;
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t v = v0 + j * stride;
      if (v >= n) continue;
      if (G > 1) l[j] -= (int32_t)st->voff[graph_of(st->voff, G, v)];
      st->labels[v] = l[j];
    }
  }
}

// ---- exact forest weight ---------------------------------------------------
// float32: bins[b] accumulates the signed 24-bit significands of the weights
// whose (denormal-adjusted) biased exponent is b, so weight = sig * 2^(b-150);
// bin 0 counts +inf and bin 255 counts -inf.  uint32: bin 0 is the sum.
__device__ __forceinline__ void weight_bin(uint32_t ordw, int wtype, int *bin, long long *val) {
  if (wtype == MSF_U32) {
    *bin = 0;
    *val = (long long)ordw;
    return;
  }
  const uint32_t bits = (ordw & 0x80000000u) ? (ordw & 0x7fffffffu) : ~ordw;
  const uint32_t E = (bits >> 23) & 0xffu, M = bits & 0x7fffffu;
  const bool neg = bits >> 31;
  if (E == 255u) {
    *bin = neg ? 255 : 0;
    *val = 1;
    return;
  }
  const long long sig = E ? (long long)(M | 0x800000u) : (long long)M;
  *bin = E ? (int)E : 1;
  *val = neg ? -sig : sig;
}

// The edge mask from the forest's keys, once after the loop.  With the
// bitmap (a full compute): one bit per forest edge (the bitmap, m / 8
// bytes, stays mostly in L2), then k_mask_expand writes every mask byte in
// one coalesced pass -- a byte written per forest edge straight into a mask
// larger than L2 costs a read of its sector from DRAM (R-MAT 26: 1.36 ms).
// Without it (msf_apply_round, whose caller's mask accumulates over calls):
// one byte written per forest edge.
__global__ void __launch_bounds__(BT) k_mask_from_keys(DevState *st) {
  uint8_t *mask = st->mask;
  if (!mask) return;
  uint32_t *bits = st->mbits;
  const int64_t nm = (int64_t)st->n_msf;
  const uint64_t *keys = st->msf_keys;
  const int64_t stride = stride64();
  // UNR keys per thread and step, loaded before the stores
  for (int64_t i0 = tid64(); i0 < nm; i0 += UNR * stride) {
    uint32_t e[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) e[j] = i0 + j * stride < nm ? (uint32_t)__ldcs(keys + i0 + j * stride) : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      if (e[j] == 0xffffffffu) continue;
      if (bits) atomicOr(bits + (e[j] >> 5), 1u << (e[j] & 31u));
      else mask[e[j]] = 1;
    }
  }
}

// 16 mask bytes from 16 bits: byte j = bit j (each nibble spread to the low
// bits of four bytes by one multiplication: its copies at shifts 0, 7, 14
// and 21 do not overlap, and bit j of the nibble lands on bit 8j).
__device__ __forceinline__ uint4 spread16(uint32_t v) {
  constexpr uint32_t MUL = 0x00204081u, LOW = 0x01010101u;
  return make_uint4(((v & 0xfu) * MUL) & LOW, (((v >> 4) & 0xfu) * MUL) & LOW, (((v >> 8) & 0xfu) * MUL) & LOW,
                    (((v >> 12) & 0xfu) * MUL) & LOW);
}
// bits [e, e + 16) of the bitmap (the bitmap has a zero word past the end)
__device__ __forceinline__ uint32_t bits16(const uint32_t *bits, int64_t e) {
  const int64_t i = e >> 5;
  const uint32_t o = (uint32_t)(e & 31);
  const uint64_t w = (uint64_t)bits[i] | ((uint64_t)bits[i + 1] << 32);
  return (uint32_t)(w >> o) & 0xffffu;
}
// The mask from the bitmap: 16-byte stores between the unaligned head and
// tail of the caller's byte array, every byte written.
__global__ void __launch_bounds__(BT) k_mask_expand(DevState *st) {
  uint8_t *mask = st->mask;
  const uint32_t *bits = st->mbits;
  if (!mask || !bits) return;
  const int64_t m = st->m;
  const int64_t head = (int64_t)((16 - (reinterpret_cast<uintptr_t>(mask) & 15)) & 15);
  const int64_t h = head < m ? head : m;
  const int64_t nq = (m - h) >> 4;
  for (int64_t e = tid64(); e < h; e += stride64()) mask[e] = (uint8_t)((bits[e >> 5] >> (e & 31)) & 1u);
  uint4 *q = reinterpret_cast<uint4 *>(mask + h);
  for (int64_t i = tid64(); i < nq; i += stride64()) q[i] = spread16(bits16(bits, h + (i << 4)));
  for (int64_t e = h + (nq << 4) + tid64(); e < m; e += stride64())
    mask[e] = (uint8_t)((bits[e >> 5] >> (e & 31)) & 1u);
}

// Long accumulators of the forest weights.  One graph: the 256 bins live in
// shared memory; each thread keeps register sums for a window of SUM_WIN
// bins (ending at the largest bin among the block's first values, where the
// bulk of typical weight distributions lies; uint32 weights use bin 0 only)
// and adds the rest to shared memory, so that the many values of a few
// popular bins do not serialise on shared-memory atomics.  Batches add to
// the graph's bins in global memory.
constexpr int SUM_WIN = 8;
__global__ void __launch_bounds__(BT) k_sum(DevState *st) {
  __shared__ unsigned long long sb[256];
  __shared__ int s_top[BT / 32];
  const unsigned long long nm = st->n_msf;
  const int32_t G = st->G;
  const int wtype = st->wtype;
  if (G == 1) {
    sb[threadIdx.x] = 0;
    // window: the largest bin among the block's first values
    int b0 = 0;
    const int64_t i0 = tid64();
    if (i0 < (int64_t)nm) {
      long long v0;
      weight_bin((uint32_t)(st->msf_keys[i0] >> 32), wtype, &b0, &v0);
      if (b0 == 255) b0 = 0;  // -inf counts are not a weight bin
    }
    b0 = __reduce_max_sync(FULL, b0);
    if ((threadIdx.x & 31) == 0) s_top[threadIdx.x >> 5] = b0;
    __syncthreads();
    int top = 0;
#pragma unroll
    for (int k = 0; k < BT / 32; ++k) top = s_top[k] > top ? s_top[k] : top;
    long long acc[SUM_WIN];
#pragma unroll
    for (int j = 0; j < SUM_WIN; ++j) acc[j] = 0;
    // UNR keys per thread and step, loaded before they are summed (one
    // load in flight per thread left the pass latency-bound)
    const int64_t stride = stride64();
    for (int64_t i0 = tid64(); i0 < (int64_t)nm; i0 += UNR * stride) {
      uint32_t ow[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q)
        ow[q] = i0 + q * stride < (int64_t)nm ? (uint32_t)(__ldcs(st->msf_keys + i0 + q * stride) >> 32) : 0u;
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        if (i0 + q * stride >= (int64_t)nm) continue;
        int bin;
        long long val;
        weight_bin(ow[q], wtype, &bin, &val);
        const int d = top - bin;
        if (d >= 0 && d < SUM_WIN && bin != 0 && bin != 255) {
#pragma unroll
          for (int j = 0; j < SUM_WIN; ++j) acc[j] += (d == j) ? val : 0;
        } else if (wtype == MSF_U32) {
          acc[0] += val;  // bin 0 is the plain sum (top is 0)
        } else {
          atomicAdd(&sb[bin], (unsigned long long)val);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < SUM_WIN; ++j) {
      long long v = acc[j];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      if ((threadIdx.x & 31) == 0 && v && top - j >= 0) atomicAdd(&sb[top - j], (unsigned long long)v);
    }
    __syncthreads();
    // the block's partial accumulators (summed by k_finalize: one atomic per
    // block and bin on 256 addresses would serialise)
    st->bins[256 + (int64_t)blockIdx.x * 256 + threadIdx.x] = (long long)sb[threadIdx.x];
    return;
  }
  for (int64_t i = tid64(); i < (int64_t)nm; i += stride64()) {
    const uint64_t key = st->msf_keys[i];
    int bin;
    long long val;
    weight_bin((uint32_t)(key >> 32), wtype, &bin, &val);
    const int32_t g = graph_of(st->eoff, G, (int64_t)(uint32_t)key);
    atomicAdd(reinterpret_cast<unsigned long long *>(st->bins) + (int64_t)g * 256 + bin, (unsigned long long)val);
  }
}

// Unsigned big integer of 6 64-bit limbs.
struct Big {
  unsigned long long w[6];
};

__device__ __forceinline__ void big_add_shifted(Big &a, unsigned long long v, int sh) {
  // limbs below li get 0 with no carry; fixed trip counts keep the limbs in
  // registers
  const int li = sh >> 6, bo = sh & 63;
  const unsigned long long lo = v << bo;
  const unsigned long long hi = bo ? (v >> (64 - bo)) : 0ull;
  unsigned long long c = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const unsigned long long add = (i == li) ? lo : (i == li + 1 ? hi : 0ull);
    const unsigned long long s1 = a.w[i] + add;
    const unsigned long long c1 = s1 < add;
    const unsigned long long s2 = s1 + c;
    const unsigned long long c2 = s2 < c;
    a.w[i] = s2;
    c = c1 | c2;
  }
}

__device__ __forceinline__ int big_cmp(const Big &a, const Big &b) {
  for (int i = 5; i >= 0; --i) {
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  }
  return 0;
}

__device__ __forceinline__ void big_sub(Big &a, const Big &b) {  // a -= b, a >= b
  unsigned long long br = 0;
  for (int i = 0; i < 6; ++i) {
    const unsigned long long d1 = a.w[i] - b.w[i];
    const unsigned long long b1 = a.w[i] < b.w[i];
    const unsigned long long d2 = d1 - br;
    const unsigned long long b2 = d1 < br;
    a.w[i] = d2;
    br = b1 | b2;
  }
}


// Shifts that give 0 for shift counts of 64 or more.
__device__ __forceinline__ unsigned long long shl64(unsigned long long x, int s) { return s >= 64 ? 0ull : x << s; }
__device__ __forceinline__ unsigned long long shr64(unsigned long long x, int s) { return s >= 64 ? 0ull : x >> s; }

// Bits [lo, lo + 63] of a (lo >= 0).  Every limb is shifted into place (no
// limb is selected by a computed index, which would move a to local memory).
__device__ __forceinline__ unsigned long long big_window(const Big &a, int lo) {
  unsigned long long w = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int d = i * 64 - lo;
    w |= d >= 0 ? shl64(a.w[i], d) : shr64(a.w[i], -d);
  }
  return w;
}

// Whether any bit below position `lo` is set.
__device__ __forceinline__ bool big_any_below(const Big &a, int lo) {
  bool any = false;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const int k = lo - i * 64;  // bits of limb i below lo
    const unsigned long long mk = k >= 64 ? ~0ull : (k <= 0 ? 0ull : (1ull << k) - 1ull);
    any = any || (a.w[i] & mk) != 0;
  }
  return any;
}

// Nearest double (ties to even) of (-1)^neg * a * 2^-149.
__device__ __forceinline__ double big_to_double(const Big &a, bool neg) {
  int h = -1;
#pragma unroll
  for (int i = 5; i >= 0; --i)
    if (h < 0 && a.w[i]) h = i * 64 + 63 - __clzll((long long)a.w[i]);
  if (h < 0) return 0.0;
  unsigned long long mant;
  int e2;  // value = mant * 2^e2
  if (h <= 52) {
    mant = a.w[0];
    e2 = -149;
  } else {
    // the 64 bits ending at h: top 53 are the significand, then the round
    // bit, then 10 bits that join the sticky bits below the window
    unsigned long long w;
    bool sticky;
    if (h >= 63) {
      w = big_window(a, h - 63);
      sticky = big_any_below(a, h - 63);
    } else {
      w = a.w[0] << (63 - h);
      sticky = false;
    }
    mant = w >> 11;
    const unsigned long long rb = (w >> 10) & 1ull;
    sticky = sticky || (w & 0x3ffull);
    e2 = h - 52 - 149;
    if (rb && (sticky || (mant & 1ull))) {
      mant += 1;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        e2 += 1;
      }
    }
  }
  // normalize into [2^52, 2^53)
  while (mant < (1ull << 52)) {
    mant <<= 1;
    e2 -= 1;
  }
  const unsigned long long biased = (unsigned long long)(e2 + 52 + 1023);
  const unsigned long long bits = ((unsigned long long)neg << 63) | (biased << 52) | (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// a += b (six limbs; the sums of the accumulators stay far below 2^384)
__device__ __forceinline__ void big_add(Big &a, const Big &b) {
  unsigned long long c = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const unsigned long long s1 = a.w[i] + b.w[i];
    const unsigned long long c1 = s1 < b.w[i];
    const unsigned long long s2 = s1 + c;
    const unsigned long long c2 = s2 < c;
    a.w[i] = s2;
    c = c1 | c2;
  }
}

// Nearest double of (P - N) * 2^-149: |P - N| and its sign, one rounding;
// per-limb selects keep the limbs in registers.
__device__ __forceinline__ double round_difference(const Big &P, const Big &N) {
  const bool ge = big_cmp(P, N) >= 0;
  Big D, E;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    D.w[i] = ge ? P.w[i] : N.w[i];
    E.w[i] = ge ? N.w[i] : P.w[i];
  }
  big_sub(D, E);
  return big_to_double(D, !ge);
}

// Exact total of one graph from its long accumulators (bin 0: +inf count
// or, for u32 weights, the plain sum; bin 255: -inf count; bins 1..254:
// signed multiples of 2^(e-1)), rounded once to nearest even.
__device__ double combine_bins(const long long *b, int wtype) {
  if (wtype == MSF_U32) return __ull2double_rn((unsigned long long)b[0]);
  const bool pinf = b[0] > 0, ninf = b[255] > 0;
  if (pinf || ninf) {
    const unsigned long long bits = (pinf && ninf) ? 0x7ff8000000000000ull
                                    : (pinf ? 0x7ff0000000000000ull : 0xfff0000000000000ull);
    return __longlong_as_double((long long)bits);
  }
  Big P, N;
  for (int i = 0; i < 6; ++i) P.w[i] = N.w[i] = 0;
  for (int e = 1; e < 255; ++e) {
    const long long v = b[e];
    if (v > 0) big_add_shifted(P, (unsigned long long)v, e - 1);
    else if (v < 0) big_add_shifted(N, (unsigned long long)(-v), e - 1);
  }
  return round_difference(P, N);
}

// The same by a whole warp (every lane calls it; lane 0 gets the result):
// lane l adds bins 8l .. 8l+7 into its own pair of big integers, the pairs
// are summed across the warp, lane 0 rounds the difference once.
__device__ double combine_bins_warp(const long long *b, int wtype) {
  if (wtype == MSF_U32) return __ull2double_rn((unsigned long long)b[0]);
  const bool pinf = b[0] > 0, ninf = b[255] > 0;
  if (pinf || ninf) {
    const unsigned long long bits = (pinf && ninf) ? 0x7ff8000000000000ull
                                    : (pinf ? 0x7ff0000000000000ull : 0xfff0000000000000ull);
    return __longlong_as_double((long long)bits);
  }
  const int lane = threadIdx.x & 31;
  Big P, N;
#pragma unroll
  for (int i = 0; i < 6; ++i) P.w[i] = N.w[i] = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int e = 8 * lane + k;
    const long long v = (e >= 1 && e <= 254) ? b[e] : 0;
    if (v > 0) big_add_shifted(P, (unsigned long long)v, e - 1);
    else if (v < 0) big_add_shifted(N, (unsigned long long)(-v), e - 1);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    Big P2, N2;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      P2.w[i] = __shfl_down_sync(FULL, P.w[i], off);
      N2.w[i] = __shfl_down_sync(FULL, N.w[i], off);
    }
    if (lane + off < 32) {
      big_add(P, P2);
      big_add(N, N2);
    }
  }
  return round_difference(P, N);
}

// One warp per graph: the warp stages the graph's 256 long accumulators in
// shared memory (coalesced), then its first lane combines them exactly.
__global__ void __launch_bounds__(BT) k_finalize(DevState *st, int nparts) {
  if (!st->totals) return;
  __shared__ long long sbin[BT / 32][256];
  const int32_t G = st->G;
  if (G == 1) {
    // one graph: block 0 sums the nparts partial accumulators of k_sum bin by
    // bin (thread t: bin t), and its first warp combines them
    static_assert(BT == 256, "one thread per bin");
    if (blockIdx.x != 0) return;
    long long *sb = sbin[0];
    const long long *part = st->bins + 256;
    long long acc = 0;
#pragma unroll 8
    for (int b = 0; b < nparts; ++b) acc += part[(int64_t)b * 256 + threadIdx.x];
    sb[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      const double t = combine_bins_warp(sb, st->wtype);
      if (threadIdx.x == 0) st->totals[0] = t;
    }
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long *sb = sbin[wid];
  const int64_t nwarps = (int64_t)gridDim.x * (BT / 32);
  for (int64_t g = (int64_t)blockIdx.x * (BT / 32) + wid; g < G; g += nwarps) {
    const long long *b = st->bins + g * 256;
#pragma unroll
    for (int q = 0; q < 8; ++q) sb[lane + 32 * q] = b[lane + 32 * q];
    __syncwarp();
    if (lane == 0) st->totals[g] = combine_bins(sb, st->wtype);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(BT) k_backward(int64_t m, int32_t G, const int64_t *eoff, const uint8_t *mask,
                                                 const double *gt, float *gw) {
  for (int64_t e = tid64(); e < m; e += stride64()) {
    float v = 0.f;
    if (mask[e]) {
      const int32_t g = (G > 1) ? bsearch_off(eoff, G, e) : 0;
      v = (float)gt[g];
    }
    gw[e] = v;
  }
}

__global__ void __launch_bounds__(BT) k_check_range(const int32_t *a, int64_t n, int32_t hi, int *flag) {
  bool bad = false;
  for (int64_t i = tid64(); i < n; i += stride64()) bad |= (a[i] < 0 || a[i] >= hi);
  if (bad) atomicOr(flag, 1);
}

__global__ void __launch_bounds__(BT) k_off_table(const int64_t *off, int32_t G, int64_t total) {
  int32_t *blk = reinterpret_cast<int32_t *>(const_cast<int64_t *>(off) + G + 1);
  const int64_t nb = off_table_len(total);
  for (int64_t b = tid64(); b < nb; b += stride64()) {
    int64_t x = b << OFF_BLK;
    if (x > total - 1) x = total - 1;
    blk[b] = bsearch_off(off, G, x);
  }
}

int vgrid(int per_sm = 4) { return sm_count() * per_sm; }

}  // namespace

int sum_partials() { return vgrid(2); }
void launch_load_state(DevState *slot, const DevState &host, cudaStream_t s) {
  k_load_state<<<1, 1, 0, s>>>(slot, host);
}
void launch_init(DevState *st, cudaStream_t s) { k_init<<<vgrid(8), BT, 0, s>>>(st); }
void launch_hook(DevState *st, cudaStream_t s) {
  k_hook<<<vgrid(8), BT, 0, s>>>(st);
  k_tiebreak<<<vgrid(8), BT, 0, s>>>(st);
}
void launch_jump_init(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_jump_init<<<1, 1, 0, s>>>(st, h);
}
void launch_jump(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_jump<<<vgrid(4), BT, 0, s>>>(st);
  k_jump_end<<<1, 1, 0, s>>>(st, h);
}
void launch_shortcut_all(DevState *st, cudaStream_t s) { k_shortcut_all<<<vgrid(8), BT, 0, s>>>(st); }
void launch_starcheck(DevState *st, cudaStream_t s) {
  k_star_init<<<vgrid(8), BT, 0, s>>>(st);
  k_star_mark<<<vgrid(8), BT, 0, s>>>(st);
  k_star_pull<<<vgrid(8), BT, 0, s>>>(st);
}
void launch_short_step(DevState *st, cudaStream_t s) {
  k_short_step<<<vgrid(8), BT, 0, s>>>(st);
  k_copy_parent<<<vgrid(8), BT, 0, s>>>(st);
}
void launch_short_full(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_short_full<<<vgrid(8), BT, 0, s>>>(st);
  k_jump_end<<<1, 1, 0, s>>>(st, h);
}
void launch_cc_hook(DevState *st, cudaStream_t s) { k_cc_hook<<<vgrid(8), BT, 0, s>>>(st); }
void launch_os_decide(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_os_decide<<<1, 1, 0, s>>>(st, h);
}
void launch_round_end(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_round_end<<<1, 1, 0, s>>>(st, h);
}
void launch_compact_decide(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_compact_decide<<<1, 1, 0, s>>>(st, h);
}
void launch_labels(DevState *st, cudaStream_t s) {
  k_label_init<<<vgrid(8), BT, 0, s>>>(st);
  k_label_min<<<vgrid(8), BT, 0, s>>>(st);
  k_label_write<<<vgrid(8), BT, 0, s>>>(st);
}
void launch_sums(DevState *st, cudaStream_t s) {
  k_mask_from_keys<<<vgrid(4), BT, 0, s>>>(st);
  k_mask_expand<<<vgrid(8), BT, 0, s>>>(st);
  k_sum<<<sum_partials(), BT, 0, s>>>(st);
  k_finalize<<<vgrid(1), BT, 0, s>>>(st, sum_partials());
}
void launch_mask_from_keys(DevState *st, cudaStream_t s) { k_mask_from_keys<<<vgrid(4), BT, 0, s>>>(st); }
void launch_off_table(const int64_t *off, int32_t G, int64_t total, cudaStream_t s) {
  if (total > 0) k_off_table<<<vgrid(1), BT, 0, s>>>(off, G, total);
}
void launch_check_range(const int32_t *a, int64_t n, int32_t hi, int *flag, cudaStream_t s) {
  k_check_range<<<vgrid(4), BT, 0, s>>>(a, n, hi, flag);
}
void launch_backward(int64_t m, int32_t G, const int64_t *eoff_d, const uint8_t *mask, const double *gt,
                     float *gw, cudaStream_t s) {
  int64_t b = (m + BT - 1) / BT;
  if (b > vgrid(8)) b = vgrid(8);
  if (b < 1) b = 1;
  k_backward<<<(int)b, BT, 0, s>>>(m, G, eoff_d, mask, gt, gw);
}

}  // namespace msf

// ---- allocation-free forest weight --------------------------------------------
//
// msf_forest_weight_noalloc sums the weights of the forest edges of up to
// NOALLOC_MAX_GRAPHS graphs exactly, like the end of msf_compute, but takes
// its scratch (the long accumulators and a copy of the edge offsets) from one
// statically sized device array of this file instead of allocating it.  The
// array lives on every GPU that loads the library until the process exits.
namespace msf {
namespace {

constexpr int NOALLOC_MAX_GRAPHS = 1024;
constexpr size_t NOALLOC_BIN_BYTES = (size_t)NOALLOC_MAX_GRAPHS * 256 * sizeof(long long);
constexpr size_t NOALLOC_OFF_BYTES = (size_t)(NOALLOC_MAX_GRAPHS + 1) * sizeof(int64_t);
constexpr size_t NOALLOC_BYTES = NOALLOC_BIN_BYTES + NOALLOC_OFF_BYTES + (size_t)NOALLOC_MAX_GRAPHS * sizeof(int);

// [0, NOALLOC_BIN_BYTES): 256 long accumulators per graph; then eoff[G+1];
// then one NaN flag per graph.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

__global__ void __launch_bounds__(BT) k_na_zero(long long *bins, int *nan_flag, int32_t G) {
  for (int64_t i = tid64(); i < (int64_t)G * 256; i += stride64()) bins[i] = 0;
  for (int64_t i = tid64(); i < (int64_t)G; i += stride64()) nan_flag[i] = 0;
}

// A selected NaN weight has no place in the long accumulator (its exponent
// field would count it as an infinity): it sets the graph's flag instead.
__global__ void __launch_bounds__(BT) k_na_sum(const uint8_t *mask, const uint32_t *w, int wtype, int64_t m,
                                               int32_t G, const int64_t *eoff, long long *bins, int *nan_flag) {
  for (int64_t e = tid64(); e < m; e += stride64()) {
    if (!mask[e]) continue;
    const int32_t g = (G > 1) ? bsearch_off(eoff, G, e) : 0;
    const uint32_t wb = w[e];
    if (wtype == MSF_F32 && (wb & 0x7fffffffu) > 0x7f800000u) {
      nan_flag[g] = 1;
      continue;
    }
    int bin;
    long long val;
    weight_bin(ord_weight_dev(wb, wtype), wtype, &bin, &val);
    atomicAdd(reinterpret_cast<unsigned long long *>(bins) + (int64_t)g * 256 + bin, (unsigned long long)val);
  }
}

__global__ void k_na_finalize(const long long *bins, const int *nan_flag, int32_t G, int wtype, double *totals) {
  for (int64_t g = tid64(); g < G; g += stride64())
    totals[g] = nan_flag[g] ? __longlong_as_double(0x7ff8000000000000ll) : combine_bins(bins + g * 256, wtype);
}

bool na_is_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (host code cannot use the symbol's name as an address).  The
// cached address is valid for the life of the device's primary context: after
// cudaDeviceReset the library must not be called on that device again in the
// same process.
int na_scratch(unsigned char **out) {
  static std::mutex mu;
  static unsigned char *addr[128] = {nullptr};
  int dev = 0;
  MSF_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(MSF_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    MSF_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = (unsigned char *)p;
  }
  *out = addr[dev];
  return MSF_OK;
}

}  // namespace
}  // namespace msf

extern "C" int msf_forest_weight_noalloc(int32_t G, int64_t m, const int64_t *eoff, const uint8_t *edge_mask,
                                         const void *w, int wtype, double *totals, void *stream) {
  using namespace msf;
  set_error("");
  if (G < 1 || G > NOALLOC_MAX_GRAPHS)
    return fail(MSF_ERR_TOO_LARGE, "msf_forest_weight_noalloc handles 1 to " +
                                       std::to_string(NOALLOC_MAX_GRAPHS) + " graphs per call");
  if (m < 0 || m > 4294967294LL) return fail(MSF_ERR_INVALID_ARG, "m must be in [0, 2^32 - 2]");
  if (wtype != MSF_F32 && wtype != MSF_U32) return fail(MSF_ERR_INVALID_ARG, "wtype must be MSF_F32 or MSF_U32");
  if (!totals || (m > 0 && (!edge_mask || !w))) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  if (G > 1) {
    if (!eoff) return fail(MSF_ERR_INVALID_ARG, "eoff is required when G > 1");
    if (eoff[0] != 0 || eoff[G] != m) return fail(MSF_ERR_INVALID_ARG, "eoff[0] must be 0 and eoff[G] must be m");
    for (int32_t g = 0; g < G; ++g)
      if (eoff[g + 1] < eoff[g]) return fail(MSF_ERR_INVALID_ARG, "eoff must be non-decreasing");
  }
  if (!na_is_device(totals) || (m > 0 && (!na_is_device(edge_mask) || !na_is_device(w))))
    return fail(MSF_ERR_INVALID_ARG, "edge_mask, w and totals must be device memory (staging would allocate)");
  unsigned char *base = nullptr;
  if (int rc = na_scratch(&base)) return rc;
  long long *bins = reinterpret_cast<long long *>(base);
  int64_t *eoff_d = reinterpret_cast<int64_t *>(base + NOALLOC_BIN_BYTES);
  int *nan_flag = reinterpret_cast<int *>(base + NOALLOC_BIN_BYTES + NOALLOC_OFF_BYTES);
  cudaStream_t s = (cudaStream_t)stream;
  if (G > 1) MSF_CK(cudaMemcpyAsync(eoff_d, eoff, (size_t)(G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_na_zero<<<vgrid(2), BT, 0, s>>>(bins, nan_flag, G);
  if (m > 0) {
    int64_t b = (m + BT - 1) / BT;
    if (b > vgrid(8)) b = vgrid(8);
    k_na_sum<<<(int)b, BT, 0, s>>>(edge_mask, (const uint32_t *)w, wtype, m, G, eoff_d, bins, nan_flag);
  }
  k_na_finalize<<<(G + BT - 1) / BT, BT, 0, s>>>(bins, nan_flag, G, wtype, totals);
  MSF_CK(cudaGetLastError());
  return MSF_OK;
}

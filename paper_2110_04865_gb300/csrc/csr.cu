// CSR builder and symmetriser.
//
// From an undirected edge list (COO) the builder stores the adjacency matrix
// A of Sec. 2 (a_ij = w(i,j) if (i,j) is an edge, as in Algorithm 2) as a
// symmetric, doubly compressed CSR: one row per vertex of nonzero degree,
// both directions of every non-loop edge, each slot carrying the column and
// the 64-bit key ord(w) << 32 | e of its undirected edge e.
//
//   1. validation of indices and weights, endpoint table ends[e], count of
//      the non-loop edges;
//   2. grouping of both directions of every edge by row (radix.cu: stable
//      LSD radix passes, no atomics), rows[] and rp[] from the sorted rows;
//   3. the tile -> first-row map, the row-start marks and the padding of the
//      slot arrays.
#include <cuda/atomic>

#include "internal.cuh"

namespace msf {

namespace {

constexpr int BT = 256;


int grid_for(int64_t work, int per_sm = 8) {
  int64_t b = (work + BT - 1) / BT;
  int64_t cap = (int64_t)sm_count() * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

__global__ void __launch_bounds__(BT) k_csr_to_coo(const int64_t *row_ptr, const int32_t *col,
                                                   int64_t n, int64_t m, int32_t *src_out, int *err) {
  const int64_t stride = (int64_t)gridDim.x * BT;
  for (int64_t s = (int64_t)blockIdx.x * BT + threadIdx.x; s < m; s += stride) {
    // row of slot s: largest i with row_ptr[i] <= s
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
      int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] <= s) lo = mid; else hi = mid;
    }
    const int32_t c = col[s];
    if (c < 0 || c >= n) { atomicOr(err, 1); src_out[s] = 0; continue; }
    // slots with row >= column are not edges: make them self-loops
    src_out[s] = (lo < c) ? (int32_t)lo : c;
  }
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < n; i += stride)
    if (row_ptr[i + 1] < row_ptr[i]) atomicOr(err, 4);
}

// Validates one edge (validate_edge) and, with DEG, counts the degrees of
// both endpoints of a non-loop edge (per-vertex atomic builder).
template <bool DEG>
__device__ __forceinline__ int2 check_edge(int64_t e, int64_t u, int64_t v, uint32_t wb, int wtype, int64_t n,
                                           int32_t G, const int64_t *eoff, const int64_t *voff, int *err,
                                           unsigned &cnt, unsigned *deg) {
  const int2 uv = validate_edge(e, u, v, wb, wtype, n, G, eoff, voff, err);
  if (uv.x != uv.y) {
    ++cnt;
    if (DEG) {
      atomicAdd(deg + uv.x, 1u);  // a degree never exceeds m < 2^32 - 1
      atomicAdd(deg + uv.y, 1u);
    }
  }
  return uv;
}

// Validates the edges, writes the endpoint table (global ids) and counts the
// non-loop edges (and, with DEG, the vertex degrees).  VEC: src, dst and w
// are 16-byte aligned and every thread takes four consecutive edges per
// step with 16-byte loads and stores; the last m % 4 edges go one by one.
template <bool DEG, bool VEC>
__global__ void __launch_bounds__(BT) k_validate(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                                 const uint32_t *__restrict__ w, int wtype, int64_t m, int64_t n,
                                                 int32_t G, const int64_t *eoff, const int64_t *voff,
                                                 int2 *__restrict__ ends, int *err, unsigned long long *nonloop,
                                                 unsigned *deg) {
  const int64_t stride = (int64_t)gridDim.x * BT;
  const int64_t tid = (int64_t)blockIdx.x * BT + threadIdx.x;
  unsigned cnt = 0;
  int64_t e0 = 0;
  if (VEC) {
    const int64_t m4 = m >> 2;
    for (int64_t q = tid; q < m4; q += stride) {
      const int4 s4 = __ldcs(reinterpret_cast<const int4 *>(src) + q);
      const int4 d4 = __ldcs(reinterpret_cast<const int4 *>(dst) + q);
      const uint4 w4 = __ldg(reinterpret_cast<const uint4 *>(w) + q);  // read again by the scatter
      const int64_t e = q << 2;
      const int2 a = check_edge<DEG>(e, s4.x, d4.x, w4.x, wtype, n, G, eoff, voff, err, cnt, deg);
      const int2 b = check_edge<DEG>(e + 1, s4.y, d4.y, w4.y, wtype, n, G, eoff, voff, err, cnt, deg);
      const int2 c = check_edge<DEG>(e + 2, s4.z, d4.z, w4.z, wtype, n, G, eoff, voff, err, cnt, deg);
      const int2 d = check_edge<DEG>(e + 3, s4.w, d4.w, w4.w, wtype, n, G, eoff, voff, err, cnt, deg);
      int4 *o = reinterpret_cast<int4 *>(ends + e);
      o[0] = make_int4(a.x, a.y, b.x, b.y);
      o[1] = make_int4(c.x, c.y, d.x, d.y);
    }
    e0 = m4 << 2;
  }
  for (int64_t e = e0 + tid; e < m; e += stride)
    ends[e] = check_edge<DEG>(e, src[e], dst[e], w[e], wtype, n, G, eoff, voff, err, cnt, deg);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nonloop, (unsigned long long)cnt);
}

__global__ void k_slots_from_edges(long long *small) { small[4] = 2 * small[5]; }

// Consecutive pairs among LOCALITY_SAMPLES evenly spread edges whose sources
// or destinations lie more than `win` vertices apart (none for CSR input,
// whose rows come in order).  Where few pairs do -- a lattice listed vertex
// by vertex, a batch of small graphs listed graph by graph -- the
// per-vertex atomic cursors write within a window of the slot arrays that
// stays in L2.
constexpr int64_t LOCALITY_SAMPLES = 1 << 13;
__global__ void __launch_bounds__(BT) k_count_scattered(const int32_t *src, const int32_t *dst, int64_t m,
                                                        int64_t win, unsigned long long *out) {
  if (!src || m < 2) return;
  unsigned c = 0;
  for (int64_t k = (int64_t)blockIdx.x * BT + threadIdx.x; k + 1 < LOCALITY_SAMPLES;
       k += (int64_t)gridDim.x * BT) {
    const int64_t i = k * (m - 1) / LOCALITY_SAMPLES, j = (k + 1) * (m - 1) / LOCALITY_SAMPLES;
    const int64_t ds = (int64_t)src[i] - (int64_t)src[j], dd = (int64_t)dst[i] - (int64_t)dst[j];
    c += (ds > win || -ds > win || dd > win || -dd > win);
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

// ---- builder by per-vertex atomic counters ------------------------------------
// Degree count (atomicAdd), exclusive scans of the degrees (slot offsets) and
// of the nonzero flags (row numbers), then a scatter of both directions with
// an atomic cursor per vertex (slot order inside a row is arbitrary).  Fast
// while the per-vertex counters stay in L2; the radix builder wins beyond.
// Degrees and row numbers in one scan: every vertex contributes the packed
// value (deg > 0) << 33 | deg.  The degree sum (at most 2m < 2^33) and the
// count of nonzero degrees (at most n < 2^31) each stay inside their field,
// so the exclusive sums of the packed values hold both prefix sums.
constexpr int PACK_SHIFT = 33;
constexpr int64_t PACK_LOW = ((int64_t)1 << PACK_SHIFT) - 1;
// The per-vertex passes below take UNR vertices per thread and step, loads
// first: a grid-stride loop whose body stores before the next load keeps one
// load per thread in flight, which leaves these passes latency-bound on
// graphs with tens of millions of vertices.
constexpr int UNR = 4;

__global__ void __launch_bounds__(BT) k_row_pack(const uint32_t *__restrict__ deg32, int64_t n,
                                                 int64_t *__restrict__ packed, int64_t *n_dev) {
  const int64_t stride = (int64_t)gridDim.x * BT;
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_dev = n;  // the scan's length
  for (int64_t v0 = (int64_t)blockIdx.x * BT + threadIdx.x; v0 < n; v0 += UNR * stride) {
    uint32_t d[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) d[j] = v0 + j * stride < n ? deg32[v0 + j * stride] : 0u;
#pragma unroll
    for (int j = 0; j < UNR; ++j)
      if (v0 + j * stride < n) packed[v0 + j * stride] = ((int64_t)(d[j] > 0) << PACK_SHIFT) | (int64_t)d[j];
  }
}

// cursor[v] = start of row v's slots (the scanned packed values are
// replaced in place); rows[] and rp[] of the nonzero-degree vertices;
// small[1] = nnz and small[2] = rows from the packed total.
// PAIRED (every slot index below 2^32): cursor[v] = start << 32 | start, a
// cursor whose high half keeps the row's first slot (see k_scatter).
template <bool PAIRED>
__global__ void __launch_bounds__(BT) k_rows_write(const uint32_t *__restrict__ deg, int64_t n, int64_t *total_dev,
                                                   int32_t *__restrict__ rows, int64_t *__restrict__ rp,
                                                   int64_t *__restrict__ cursor) {
  const int64_t stride = (int64_t)gridDim.x * BT;
  for (int64_t v0 = (int64_t)blockIdx.x * BT + threadIdx.x; v0 < n; v0 += UNR * stride) {
    int64_t x[UNR];
    uint32_t d[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t v = v0 + j * stride;
      x[j] = v < n ? cursor[v] : 0;
      d[j] = v < n ? deg[v] : 0u;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t v = v0 + j * stride;
      if (v >= n) continue;
      const int64_t off = x[j] & PACK_LOW, pos = x[j] >> PACK_SHIFT;
      cursor[v] = PAIRED ? (int64_t)(((uint64_t)off << 32) | (uint64_t)off) : off;
      if (d[j] > 0) {
        rows[pos] = (int32_t)v;
        rp[pos] = off;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t t = *total_dev;
    const int64_t nnz = t & PACK_LOW, nrows = t >> PACK_SHIFT;
    rp[nrows] = nnz;
    total_dev[-1] = nnz;  // small[1]
    total_dev[0] = nrows; // small[2]
  }
}

// A claimed cursor value: the slot, and the row-start mark for it.  A
// paired cursor (start << 32 | next) returns its row's first slot with
// every claim, so the claim that receives that slot marks it; the low half
// never carries into the high one, since every slot index is below 2^32.
template <bool PAIRED>
__device__ __forceinline__ int64_t claim_slot(unsigned long long o) {
  return PAIRED ? (int64_t)(uint32_t)o : (int64_t)o;
}
template <bool PAIRED>
__device__ __forceinline__ int32_t claim_head(unsigned long long o) {
  return (PAIRED && (uint32_t)o == (uint32_t)(o >> 32)) ? (int32_t)COL_HEAD : 0;
}

template <bool PAIRED>
__device__ __forceinline__ void scatter_one(int2 uv, uint32_t wb, int wtype, int64_t e,
                                            unsigned long long *cursor, int32_t *col, uint64_t *key) {
  if (uv.x == uv.y) return;
  const uint64_t k = ((uint64_t)ord_weight_dev(wb, wtype) << 32) | (uint64_t)e;
  const unsigned long long a = atomicAdd(cursor + uv.x, 1ull);
  const unsigned long long b = atomicAdd(cursor + uv.y, 1ull);
  col[claim_slot<PAIRED>(a)] = uv.y | claim_head<PAIRED>(a);
  key[claim_slot<PAIRED>(a)] = k;
  col[claim_slot<PAIRED>(b)] = uv.x | claim_head<PAIRED>(b);
  key[claim_slot<PAIRED>(b)] = k;
}

// Both directions of every non-loop edge to the next free slot of its row.
// Four consecutive edges per thread and step (16-byte loads; w 16-byte
// aligned when VEC), so that eight cursor atomics are in flight at once.
// PAIRED: paired cursors (every slot index below 2^32); the scatter then
// sets the row-start marks itself, so the tile-map pass writes no column
// word (its read-modify-write of col touches every sector of col when rows
// are short).  Otherwise plain 64-bit cursors.
// Edges [lo, hi) (lo a multiple of four).
template <bool VEC, bool PAIRED>
__global__ void __launch_bounds__(BT) k_scatter(const int2 *__restrict__ ends, const uint32_t *__restrict__ w,
                                                int wtype, int64_t lo, int64_t hi, unsigned long long *cursor,
                                                int32_t *__restrict__ col, uint64_t *__restrict__ key) {
  const int64_t stride = (int64_t)gridDim.x * BT;
  const int64_t tid = (int64_t)blockIdx.x * BT + threadIdx.x;
  int64_t e0 = lo;
  if (VEC) {
    const int64_t m4 = hi >> 2;
    for (int64_t q = (lo >> 2) + tid; q < m4; q += stride) {
      const int4 p0 = __ldcs(reinterpret_cast<const int4 *>(ends) + 2 * q);
      const int4 p1 = __ldcs(reinterpret_cast<const int4 *>(ends) + 2 * q + 1);
      const uint4 w4 = __ldcs(reinterpret_cast<const uint4 *>(w) + q);
      const int64_t e = q << 2;
      const uint64_t k0 = ((uint64_t)ord_weight_dev(w4.x, wtype) << 32) | (uint64_t)e;
      const uint64_t k1 = ((uint64_t)ord_weight_dev(w4.y, wtype) << 32) | (uint64_t)(e + 1);
      const uint64_t k2 = ((uint64_t)ord_weight_dev(w4.z, wtype) << 32) | (uint64_t)(e + 2);
      const uint64_t k3 = ((uint64_t)ord_weight_dev(w4.w, wtype) << 32) | (uint64_t)(e + 3);
      // cursor atomics first (independent), then the eight slot writes.
      // Edge lists with row locality list a vertex's edges together (a
      // lattice or a geometric graph listed vertex by vertex): a run of
      // consecutive edges with the same first endpoint takes its slots in
      // that row with one atomic.
      unsigned long long s[8];
      const bool l0 = p0.x != p0.y, l1 = p0.z != p0.w, l2 = p1.x != p1.y, l3 = p1.z != p1.w;
      const bool c1 = l0 && l1 && p0.z == p0.x;  // edge 1 continues edge 0's run
      const bool c2 = l1 && l2 && p1.x == p0.z;
      const bool c3 = l2 && l3 && p1.z == p1.x;
      const unsigned n0 = 1u + (c1 ? 1u + (c2 ? 1u + (c3 ? 1u : 0u) : 0u) : 0u);
      const unsigned n1 = 1u + (c2 ? 1u + (c3 ? 1u : 0u) : 0u);
      const unsigned n2 = 1u + (c3 ? 1u : 0u);
      if (l0) s[0] = atomicAdd(cursor + p0.x, (unsigned long long)n0);
      if (l1 && !c1) s[2] = atomicAdd(cursor + p0.z, (unsigned long long)n1);
      if (l2 && !c2) s[4] = atomicAdd(cursor + p1.x, (unsigned long long)n2);
      if (l3 && !c3) s[6] = atomicAdd(cursor + p1.z, 1ull);
      if (l0) s[1] = atomicAdd(cursor + p0.y, 1ull);
      if (l1) s[3] = atomicAdd(cursor + p0.w, 1ull);
      if (l2) s[5] = atomicAdd(cursor + p1.y, 1ull);
      if (l3) s[7] = atomicAdd(cursor + p1.w, 1ull);
      // a run's later slots follow its first (never a row start: the low
      // half of the claimed value is then above the row's first slot)
      if (c1) s[2] = s[0] + 1;
      if (c2) s[4] = s[2] + 1;
      if (c3) s[6] = s[4] + 1;
#define MSF_PUT(i, c, k)                                        \
  {                                                            \
    const int64_t at = claim_slot<PAIRED>(s[i]);               \
    col[at] = (c) | claim_head<PAIRED>(s[i]);                  \
    key[at] = (k);                                             \
  }
      if (l0) { MSF_PUT(0, p0.y, k0) MSF_PUT(1, p0.x, k0) }
      if (l1) { MSF_PUT(2, p0.w, k1) MSF_PUT(3, p0.z, k1) }
      if (l2) { MSF_PUT(4, p1.y, k2) MSF_PUT(5, p1.x, k2) }
      if (l3) { MSF_PUT(6, p1.w, k3) MSF_PUT(7, p1.z, k3) }
#undef MSF_PUT
    }
    e0 = (m4 << 2) > lo ? (m4 << 2) : lo;
  }
  for (int64_t e = e0 + tid; e < hi; e += stride)
    scatter_one<PAIRED>(ends[e], w[e], wtype, e, cursor, col, key);
}

// tile_row[b] = row containing slot b*TB for b*TB < nnz, nrows beyond; the
// first slot of every row gets the COL_HEAD mark (unless `marked`: the
// builder has set them); slots
// [nnz, roundup(nnz, SLOT_PAD)) are padded with (col 0, key KEY_INF).
__device__ void fill_tile_rows(const int64_t *__restrict__ rp, int64_t nrows, int64_t nnz,
                               int32_t *__restrict__ tile_row, int32_t *col, uint64_t *key, bool marked = false) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t padded = (nnz + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD;
  for (int64_t k0 = tid; k0 <= nrows; k0 += UNR * stride) {
    int64_t a[UNR], e[UNR];
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t k = k0 + j * stride;
      a[j] = k < nrows ? rp[k] : nnz;
      e[j] = k < nrows ? rp[k + 1] : nnz;
    }
#pragma unroll
    for (int j = 0; j < UNR; ++j) {
      const int64_t k = k0 + j * stride;
      if (k > nrows) continue;
      int64_t b0, b1;
      if (k < nrows) {
        b0 = (a[j] + TB - 1) / TB;
        b1 = (e[j] + TB - 1) / TB;
        if (!marked) col[a[j]] |= (int32_t)COL_HEAD;  // row start mark
      } else {
        b0 = (nnz + TB - 1) / TB;
        b1 = padded / TB + 1;
      }
      for (int64_t b = b0; b < b1; ++b) tile_row[b] = (int32_t)k;
    }
  }
  for (int64_t s = nnz + tid; s < padded; s += stride) {
    col[s] = 0;
    key[s] = KEY_INF;
  }
}

__global__ void __launch_bounds__(BT) k_tile_rows_explicit(const int64_t *rp, const int64_t *nrows_dev,
                                                           const int64_t *nnz_dev, int32_t *tile_row,
                                                           int32_t *col, uint64_t *key, bool marked) {
  fill_tile_rows(rp, *nrows_dev, *nnz_dev, tile_row, col, key, marked);
}

__global__ void __launch_bounds__(BT) k_tile_rows_state(DevState *st, int which) {
  const int b = which < 0 ? st->cur : which;
  const CsrBuf &B = st->buf[b];
  fill_tile_rows(B.rp, st->nrows, st->nnz, B.tile_row, B.col, B.key);
}

// Scratch blocks of one call, returned to the pool behind the work queued on
// the stream (or at once when no stream is given).
struct Tmp {
  void *p[8] = {nullptr};
  int k = 0;
  cudaStream_t s = nullptr;
  bool ordered = false;
  Tmp() = default;
  explicit Tmp(cudaStream_t st) : s(st), ordered(true) {}
  void *get(size_t bytes, int *err) {
    void *q = pool_alloc(bytes, err);
    p[k++] = q;
    return q;
  }
  ~Tmp() {
    for (int i = 0; i < k; ++i) {
      if (ordered) pool_free_after(p[i], s);
      else pool_free(p[i]);
    }
  }
};

}  // namespace

// Rows of nonzero degree from the vertex degrees: rows[], rp[] (slot
// offsets), small[1] = nnz, small[2] = nrows, and cursor[v] = rp of v's row
// (the first free slot of v, for the scatter).  `cursor` has n + 1 entries.
// paired: cursor[v] = start << 32 | start instead (every slot index below 2^32)
static int rows_from_degrees_impl(int64_t n, const uint32_t *deg, long long *small, CsrBuf &csr,
                                  int64_t *cursor, cudaStream_t s, bool paired) {
  int err = MSF_OK;
  Tmp tmp(s);
  int64_t *scan_tmp = (int64_t *)tmp.get((size_t)(NB_SCAN + 1) * 8, &err);
  if (err) return err;
  int64_t *nv = (int64_t *)tmp.get(64, &err);
  if (err) return err;
  k_row_pack<<<grid_for(n), BT, 0, s>>>(deg, n, cursor, nv);
  // the packed total lands in small[2]; k_rows_write splits it into small[1..2]
  launch_scan_excl(cursor, cursor, nv, scan_tmp, (int64_t *)(small + 2), s);
  if (paired) k_rows_write<true><<<grid_for(n), BT, 0, s>>>(deg, n, (int64_t *)(small + 2), csr.rows, csr.rp, cursor);
  else k_rows_write<false><<<grid_for(n), BT, 0, s>>>(deg, n, (int64_t *)(small + 2), csr.rows, csr.rp, cursor);
  MSF_CK(cudaGetLastError());
  return MSF_OK;
}

int rows_from_degrees(int64_t n, const uint32_t *deg, long long *small, CsrBuf &csr, int64_t *cursor,
                      cudaStream_t s) {
  return rows_from_degrees_impl(n, deg, small, csr, cursor, s, false);
}

// `deg` holds the degrees counted by k_validate<true>.  *marked is set when
// the scatter has written the row-start marks (paired cursors).
int atomic_build_csr(int64_t n, int64_t m, const int2 *ends, const uint32_t *w, int wtype, long long *small,
                     const uint32_t *deg, CsrBuf &csr, cudaStream_t s, bool *marked) {
  int err = MSF_OK;
  Tmp tmp(s);
  int64_t *cursor = (int64_t *)tmp.get((size_t)(n + 1) * 8, &err);
  if (err) return err;
  // paired cursors while every slot index (< 2m) fits in 32 bits
  const bool paired = 2 * m < ((int64_t)1 << 32);
  *marked = paired;
  if (int rc = rows_from_degrees_impl(n, deg, small, csr, cursor, s, paired)) return rc;
  if (m > 0) {
    const bool vec = (reinterpret_cast<uintptr_t>(w) & 15) == 0;
    auto *cur = (unsigned long long *)cursor;
    // 2^22 edges per launch: a persistent grid drifts over many times its
    // width of the edge list, and the rows its cursors and slot writes touch
    // then fall out of L2 (measured: the 4096-graph batch's scatter hit L2
    // for 46 % of its sectors in one launch); launches over bounded ranges
    // keep them resident
    const int64_t chunk = (int64_t)1 << 22;
    for (int64_t lo = 0; lo < m; lo += chunk) {
      const int64_t hi = lo + chunk < m ? lo + chunk : m;
      const int gr = grid_for(hi - lo);
      if (paired && vec) k_scatter<true, true><<<gr, BT, 0, s>>>(ends, w, wtype, lo, hi, cur, csr.col, csr.key);
      else if (paired) k_scatter<false, true><<<gr, BT, 0, s>>>(ends, w, wtype, lo, hi, cur, csr.col, csr.key);
      else if (vec) k_scatter<true, false><<<gr, BT, 0, s>>>(ends, w, wtype, lo, hi, cur, csr.col, csr.key);
      else k_scatter<false, false><<<gr, BT, 0, s>>>(ends, w, wtype, lo, hi, cur, csr.col, csr.key);
    }
  }
  MSF_CK(cudaGetLastError());
  return MSF_OK;
}

void launch_tile_rows(DevState *st, int which, cudaStream_t s) {
  k_tile_rows_state<<<(int)sm_count() * 4, BT, 0, s>>>(st, which);
}

// Builds g->csr0 and g->ends on the device from device-resident inputs.
// `src` is ignored when row_ptr != NULL.  Synchronizes `s`.
int build_csr_device(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const int64_t *row_ptr, const void *w, int wtype, int32_t G,
                     const int64_t *eoff_d, const int64_t *voff_d, cudaStream_t s,
                     msf_graph *g) {
  int err = MSF_OK;
  Tmp tmp;
  const int64_t cap_slots = 2 * m;
  const int64_t padded = (cap_slots + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD + SLOT_PAD;
  g->ends = (int2 *)pool_alloc((size_t)(m > 0 ? m : 1) * sizeof(int2), &err);
  if (err) return err;
  g->csr0.rows = (int32_t *)pool_alloc((size_t)(n + 1) * sizeof(int32_t), &err);
  if (err) return err;
  g->csr0.rp = (int64_t *)pool_alloc((size_t)(n + 2) * sizeof(int64_t), &err);
  if (err) return err;
  g->csr0.col = (int32_t *)pool_alloc((size_t)padded * sizeof(int32_t), &err);
  if (err) return err;
  g->csr0.key = (uint64_t *)pool_alloc((size_t)padded * sizeof(uint64_t), &err);
  if (err) return err;
  g->csr0.tile_row = (int32_t *)pool_alloc((size_t)(padded / TB + 2) * sizeof(int32_t), &err);
  if (err) return err;
  g->csr0.cap_slots = cap_slots;
  g->csr0.cap_rows = n;

  // scratch: sizes and the error word
  long long *small = (long long *)tmp.get(64, &err);  // [1] nnz, [2] nrows, [3] err, [4] slots, [5] edges
  if (err) return err;
  int32_t *coo_src = nullptr;
  if (row_ptr) {
    coo_src = (int32_t *)tmp.get((size_t)(m > 0 ? m : 1) * sizeof(int32_t), &err);
    if (err) return err;
  }
  // builder (measured on GB300): bucketed from 2^20 edges (R-MAT scale 20
  // and 26, the uniform graph) unless the edge list has locality (the 256^3
  // grid, a batch of small graphs, CSR input: per-vertex atomic cursors then
  // write within an L2-sized window); per-vertex atomics for small graphs;
  // radix on request
  const int mode = options().build_mode;
  const bool radix = mode == 2;
  bool bucket = !radix && bucket_build_fits(n) && mode == 3;
  if (mode == 0 && m >= ((int64_t)1 << 20) && bucket_build_fits(n)) {
    // window: the vertices whose slots (12 bytes each, 2m / n per vertex on
    // average) fill a quarter of L2
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) {
      cudaGetLastError();
      l2 = 64 << 20;
    }
    const double per_vertex = 12.0 * 2.0 * (double)m / (double)(n > 0 ? n : 1);
    const int64_t win = (int64_t)((double)l2 / 4.0 / per_vertex) + 1;
    unsigned long long *cnt = (unsigned long long *)tmp.get(64, &err);
    if (err) return err;
    MSF_CK(cudaMemsetAsync(cnt, 0, 8, s));
    k_count_scattered<<<64, BT, 0, s>>>(row_ptr ? nullptr : src, dst, m, win, cnt);
    unsigned long long far = 0;
    MSF_CK(cudaMemcpyAsync(&far, cnt, 8, cudaMemcpyDeviceToHost, s));
    MSF_CK(cudaStreamSynchronize(s));
    bucket = far > (unsigned long long)(LOCALITY_SAMPLES / 16);
  }
  uint32_t *deg = nullptr;
  if (!radix && !bucket) {
    deg = (uint32_t *)tmp.get((size_t)(n + 1) * 4, &err);
    if (err) return err;
    MSF_CK(cudaMemsetAsync(deg, 0, (size_t)(n + 1) * 4, s));
  }
  MSF_CK(cudaMemsetAsync(small, 0, 64, s));
  int *errw = (int *)(small + 3);
  if (row_ptr) {
    k_csr_to_coo<<<grid_for(m), BT, 0, s>>>(row_ptr, dst, n, m, coo_src, errw);
    src = coo_src;
  }
  if (m > 0 && !bucket) {  // (the bucketed builder validates in its first pass)
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
                       reinterpret_cast<uintptr_t>(w)) & 15) == 0;
    auto *nl = (unsigned long long *)(small + 5);
    const uint32_t *wu = (const uint32_t *)w;
    const int gb = grid_for(vec ? (m + 3) / 4 : m);
    if ((radix || bucket) && vec)
      k_validate<false, true><<<gb, BT, 0, s>>>(src, dst, wu, wtype, m, n, G, eoff_d, voff_d, g->ends, errw, nl, deg);
    else if (radix || bucket)
      k_validate<false, false><<<gb, BT, 0, s>>>(src, dst, wu, wtype, m, n, G, eoff_d, voff_d, g->ends, errw, nl, deg);
    else if (vec)
      k_validate<true, true><<<gb, BT, 0, s>>>(src, dst, wu, wtype, m, n, G, eoff_d, voff_d, g->ends, errw, nl, deg);
    else
      k_validate<true, false><<<gb, BT, 0, s>>>(src, dst, wu, wtype, m, n, G, eoff_d, voff_d, g->ends, errw, nl, deg);
  }
  if (radix) k_slots_from_edges<<<1, 1, 0, s>>>(small);
  MSF_CK(cudaGetLastError());
  int rc;
  bool marked = false;  // row-start marks already written by the builder
  if (radix) {
    rc = radix_build_csr(n, m, g->ends, (const uint32_t *)w, wtype, small + 4, small + 2, g->csr0, s);
    if (rc) return rc;
    MSF_CK(cudaMemcpyAsync(small + 1, small + 4, 8, cudaMemcpyDeviceToDevice, s));
  } else if (bucket) {
    rc = bucket_build_csr(n, m, src, dst, (const uint32_t *)w, wtype, G, eoff_d, voff_d, g->ends, small, g->csr0, s);
    if (rc) return rc;
  } else {
    rc = atomic_build_csr(n, m, g->ends, (const uint32_t *)w, wtype, small, deg, g->csr0, s, &marked);
    if (rc) return rc;
  }
  k_tile_rows_explicit<<<grid_for(n + 1, 4), BT, 0, s>>>(g->csr0.rp, (const int64_t *)(small + 2),
                                                         (const int64_t *)(small + 1), g->csr0.tile_row,
                                                         g->csr0.col, g->csr0.key, marked);
  MSF_CK(cudaGetLastError());
  long long hsmall[4] = {0, 0, 0, 0};
  MSF_CK(cudaMemcpyAsync(hsmall, small, sizeof(hsmall), cudaMemcpyDeviceToHost, s));
  MSF_CK(cudaStreamSynchronize(s));
  const int e = (int)(hsmall[3] & 0xffffffff);
  if (e & 1) return fail(MSF_ERR_INVALID_ARG, "vertex index out of range");
  if (e & 2) return fail(MSF_ERR_INVALID_ARG, "NaN weight");
  if (e & 4) return fail(MSF_ERR_INVALID_ARG, "row_ptr is not non-decreasing");
  g->nnz0 = hsmall[1];
  g->nrows0 = hsmall[2];
  // kernels launched above: the locality sample, validation (and the slot
  // count for radix), the builder's own, the tile map (scans are three
  // launches each)
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
  const int passes = bits <= 10 ? 1 : (bits + 9) / 10;
  int builder;
  if (bucket) {
    // validate+count, scan (3), scatter, item lists, item maps, degree,
    // rows (5), place; beyond 2^22 vertices the sub-bucket pass: chunk list,
    // chunk map, count, length, scan (3), scatter, starts, and the item
    // lists as counts + two scans (3 each) instead of one launch
    builder = 14 + (bits > 22 ? 9 + 6 : 0);
  }
  else if (radix) builder = (m > 0 ? 1 : 0) + 7 + 5 * passes;  // validate; 2 sets, row bounds (5), passes
  else builder = (m > 0 ? 1 + (int)((m + ((int64_t)1 << 22) - 1) >> 22) : 0) + 5;  // validate, scatter per
                                                                              // 2^22 edges; rows (5)
  g->stats.builder = bucket ? 3 : (radix ? 2 : 1);
  g->build_kernels = (row_ptr ? 1 : 0) + (radix ? 1 : 0) /* slot count */ + builder + 1 /* tile map */ +
                     ((mode == 0 && m >= ((int64_t)1 << 20) && bucket_build_fits(n)) ? 1 : 0);
  return MSF_OK;
}

}  // namespace msf

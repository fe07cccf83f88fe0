// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "msf.h"

namespace msf {

constexpr uint64_t KEY_INF = 0xFFFFFFFFFFFFFFFFull;  // MinWeight identity
constexpr int TB = 128;        // granularity of the tile -> first-row map (slots)
constexpr int SLOT_PAD = 512;  // slot arrays are padded to a multiple of this
constexpr int NB_SCAN = 1024;  // blocks of the device-wide scans
constexpr uint32_t COL_HEAD = 0x80000000u;

// One doubly compressed CSR (only rows of nonzero degree).
//   rows[k]      vertex of row k (after compaction: a root that stands for it)
//   rp[k]        first slot of row k, rp[nrows] = nnz
//   col[s]       column vertex of slot s
//   key[s]       ord(w) << 32 | edge id
//   tile_row[b]  row containing slot b*TB (b*TB < nnz), else nrows
// Bit 31 of col[s] is set when s is the first slot of its row (COL_HEAD).
// Slots [nnz, padded) hold col = 0, key = KEY_INF.
struct CsrBuf {
  int32_t *rows;
  int64_t *rp;
  int32_t *col;
  uint64_t *key;
  int32_t *tile_row;
  int64_t cap_slots;  // capacity excluding padding
  int64_t cap_rows;
};

// Device-resident state of one computation.  Kernels captured in the CUDA
// graph receive a pointer to it and read sizes and buffers from it, so the
// same instantiated graph serves every graph computed on a stream.
struct DevState {
  // problem
  int64_t n, m;
  int32_t G, wtype;
  const int64_t *voff, *eoff;  // device [G+1] (NULL when G == 1)
  const int2 *ends;            // [m] endpoints (global ids)
  CsrBuf buf[3];               // 0 = as built (read only), 1 and 2 = compaction targets
  // current edge list
  int32_t cur;
  int32_t pad0;
  int64_t nrows, nnz;
  // vertex state
  int32_t *p;         // parent vector
  int32_t *tgt;       // hook target of each listed root; label scratch
  uint64_t *r;        // projected minimum key per root (MinWeight)
  // roots that may hook (complete shortcutting): the CSR rows at first, then
  // the roots that did not hook; every vertex under the original schedule
  const int32_t *rl;
  int32_t *rl_next;
  int32_t *rl_buf[2];
  unsigned long long rl_n, rl_next_n;
  int32_t rl_all;
  int32_t pad3;
  int64_t nrows0;     // rows of the CSR as built (buf[0])
  int32_t prow_valid; // prow holds p of the current rows (written by the shortcut pass)
  int32_t pad4;
  int32_t *changed;   // roots whose parent changed this round (Algorithm 3)
  uint64_t *msf_keys; // keys of the forest edges, in hooking order
  // compaction scratch
  int64_t *rowcnt;    // live slots per row
  int64_t *rowflag;   // row kept (1/0), scanned in place
  int64_t *tilecnt;   // live slots per min-edge tile, scanned in place
  int64_t *scan_tmp;  // NB_SCAN * 2 partials + total
  // sums
  long long *bins;    // [G * 256] long accumulator per graph
  // outputs (device)
  uint8_t *mask;
  int32_t *labels;
  double *totals;
  uint32_t *mbits;    // the forest's edges as a bitmap ((m + 31) / 32 + 2 words), expanded into mask
  // per-round counters
  unsigned long long n_hooks, n_changed, n_msf, n_live;
  unsigned long long jump_dirty;
  unsigned int ticket;
  int32_t round, jumps, status;
  int32_t compactions;
  int32_t jumps_total;
  // options
  int32_t round_limit, jump_limit;
  float tau;
  int32_t spl;        // slots per lane of the min-edge sweep
  // nonzero: p is the identity (first round), the sweep skips the gathers
  int32_t first_round_identity;
  // compaction: lengths of the scans and their totals
  int64_t scan_n[2];    // [0] min-edge tiles, [1] rows
  int64_t scan_tot[3];  // [0] live slots, [1] new nnz, [2] new rows
  // loop control: the kernels that end a loop body or decide a branch write
  // their decision here, and pass it to the CUDA graph when use_graph != 0
  int32_t use_graph;
  int32_t ctl_round, ctl_jump, ctl_compact;
  // shortcut schedule (MSF_OPT_SHORTCUT) and its data
  int32_t shortcut_mode;
  int32_t pad1;
  int64_t os_threshold;
  uint8_t *star;                  // star flags (original schedule only, else NULL)
  unsigned long long n_short;     // vertices moved by the last shortcut step
  int32_t *pjs;                   // pairwise formulation: p of every slot's column
  int32_t *colr;                  // relabelled column words of buf[0] (the second round's sweep
                                  // writes them, the later rounds read them), or NULL
  int32_t *prow;                  // p of every row of the current edge list
  unsigned long long n_active;    // roots with an outgoing edge this round
  int32_t early_stop;             // skip the confirming last round when possible
  int32_t combine;                // the next sweeps' projection goes through the block combining
                                  // table (few distinct roots: set at the end of a round)
  int32_t pad2;
};

// Order-preserving map of a weight word to an unsigned key half (-0 as +0).
__device__ __forceinline__ uint32_t ord_weight_dev(uint32_t b, int wtype) {
  if (wtype != MSF_F32) return b;
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// ---- batch offsets ------------------------------------------------------------------
// A batch's device offset arrays (vertex and edge offsets, G + 1 entries,
// non-decreasing, off[G] = the total) are followed by an int32 table:
// blk[b] = the graph of id min(b << OFF_BLK, off[G] - 1), for
// b <= ((off[G] - 1) >> OFF_BLK) + 1.  An id's graph then lies in
// [blk[b], blk[b + 1]] for b = id >> OFF_BLK: a short search instead of one
// over all G graphs for every edge, vertex and forest key.
constexpr int OFF_BLK = 12;
__host__ __device__ inline int64_t off_table_len(int64_t total) {
  return total > 0 ? ((total - 1) >> OFF_BLK) + 2 : 0;
}

// graph of id e: the g with off[g] <= e < off[g+1] (off with its table)
__device__ __forceinline__ int32_t graph_of(const int64_t *off, int32_t G, int64_t e) {
  const int32_t *blk = reinterpret_cast<const int32_t *>(off + G + 1);
  const int64_t b = e >> OFF_BLK;
  int32_t lo = blk[b], hi = blk[b + 1] + 1;  // answer in [lo, hi)
  if (hi > G) hi = G;
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}
void launch_off_table(const int64_t *off, int32_t G, int64_t total, cudaStream_t s);

// ---- edge validation (builders) ---------------------------------------------------

// Validates one edge: returns its global endpoints, or the self-loop (0, 0)
// for an invalid edge (index out of range: err |= 1; NaN weight: err |= 2),
// so that no later kernel writes through its indices.
__device__ __forceinline__ int2 validate_edge(int64_t e, int64_t u, int64_t v, uint32_t wb, int wtype, int64_t n,
                                              int32_t G, const int64_t *eoff, const int64_t *voff, int *err) {
  int64_t lim = n, base = 0;
  if (G > 1) {
    const int32_t g = graph_of(eoff, G, e);
    base = voff[g];
    lim = voff[g + 1] - base;
  }
  const bool in_range = u >= 0 && v >= 0 && u < lim && v < lim;
  const bool nan = wtype == MSF_F32 && (wb & 0x7fffffffu) > 0x7f800000u;
  if (!in_range) atomicOr(err, 1);
  if (nan) atomicOr(err, 2);
  if (!in_range || nan) return make_int2(0, 0);
  return make_int2((int)(u + base), (int)(v + base));
}

// ---- error reporting --------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define MSF_CK(call)                                      \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::msf::cuda_fail(_e, #call); \
  } while (0)

// ---- caching allocator (pool.cu) ----------------------------------------------
void *pool_alloc(size_t bytes, int *err);  // err = MSF_OK / MSF_ERR_OOM
// Returns p to the cache once the work queued on s so far has completed (no
// host synchronisation).
void pool_free_after(void *p, cudaStream_t s);
void pool_free(void *p);
void pool_release_all();

// ---- device properties ---------------------------------------------------------
int sm_count();

// ---- options ---------------------------------------------------------------------
struct Options {
  double tau = 0.5;
  int round_limit = 64;
  int jump_limit = 64;
  int spl = 4;
  int blocks_per_sm = 4;
  int prefetch = 0;
  int exec_mode = 0;  // 0 = CUDA graph, 1 = host-driven loop (profiling)
  int shortcut_mode = 0;  // MSF_SHORTCUT_* of msf.h
  int pairwise = 0;       // MSF_OPT_KERNEL
  int build_mode = 0;     // MSF_OPT_BUILD
  int early_stop = 1;     // MSF_OPT_EARLY_STOP
  int sweep = 0;          // MSF_OPT_SWEEP
  int host_input = 0;     // MSF_OPT_HOST_INPUT
  int relabel = 1;        // MSF_OPT_RELABEL
  int64_t os_threshold = 1310720;
};
Options &options();

// ---- launchers (each enqueues on `s`; sizes come from device memory where noted)
// A `DevState *st` argument is a DEVICE address: launchers may form field
// addresses from it (&st->x) but never read through it.
// scan.cu: exclusive scans of int64 arrays; N read from *n_dev (device).  The
// total is written to *total_dev.  In place allowed.
void launch_scan_excl(const int64_t *in, int64_t *out, const int64_t *n_dev, int64_t *tmp,
                      int64_t *total_dev, cudaStream_t s);
// The same, in place, with the array and scratch pointers read from device
// memory (addresses of DevState fields); nothing is dereferenced on the host.
void launch_scan_excl_ind(int64_t *const *inout_ind, const int64_t *n_dev, int64_t *const *tmp_ind,
                          int64_t *total_dev, cudaStream_t s);

// csr.cu
int build_csr_device(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const int64_t *row_ptr, const void *w, int wtype, int32_t G,
                     const int64_t *eoff_d, const int64_t *voff_d, cudaStream_t s,
                     msf_graph *g);
void launch_tile_rows(DevState *st, int which, cudaStream_t s);

// Rows of nonzero degree from the vertex degrees (csr.rows, csr.rp, small[1]
// = nnz, small[2] = nrows) and cursor[v] = first slot of v's row.
int rows_from_degrees(int64_t n, const uint32_t *deg, long long *small, CsrBuf &csr, int64_t *cursor,
                      cudaStream_t s);

// bucket.cu
bool bucket_build_fits(int64_t n);
// Validates the edges (writes ends, small[3] error bits, small[5] non-loop
// edges) and builds csr; small[1] = nnz, small[2] = nrows.
int bucket_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *w, int wtype,
                     int32_t G, const int64_t *eoff_d, const int64_t *voff_d, int2 *ends, long long *small,
                     CsrBuf &csr, cudaStream_t s);

// radix.cu
int radix_build_csr(int64_t n, int64_t m, const int2 *ends, const uint32_t *w, int wtype,
                    const long long *nslots_dev, long long *nrows_dev, CsrBuf &csr, cudaStream_t s);

// minedge.cu
// The sweep reads prow (p of every row): launch_prow must run after the last
// change of p and before the sweep (use_star: rows outside stars get -1).
void launch_prow(DevState *st, int use_star, cudaStream_t s);
void launch_min_edge(DevState *st, int spl, int blocks_per_sm, int prefetch, cudaStream_t s, int pairwise = 0);
void launch_compact(DevState *st, int spl, int blocks_per_sm, cudaStream_t s);

// rounds.cu
void launch_init(DevState *st, cudaStream_t s);
// blocks of the single-graph sum kernel: bins holds 256 accumulators for the
// graph, then one row of 256 partials per block
int sum_partials();
void launch_hook(DevState *st, cudaStream_t s);
void launch_jump_init(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_jump(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_shortcut_all(DevState *st, cudaStream_t s);
void launch_starcheck(DevState *st, cudaStream_t s);
void launch_short_step(DevState *st, cudaStream_t s);
void launch_short_full(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_os_decide(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_cc_hook(DevState *st, cudaStream_t s);
void launch_cc_sweep(DevState *st, bool conditional, cudaStream_t s);
void launch_round_end(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_compact_decide(DevState *st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_labels(DevState *st, cudaStream_t s);
void launch_sums(DevState *st, cudaStream_t s);
void launch_mask_from_keys(DevState *st, cudaStream_t s);
void launch_load_state(DevState *slot, const DevState &host, cudaStream_t s);
void launch_backward(int64_t m, int32_t G, const int64_t *eoff_d, const uint8_t *mask,
                     const double *gt, float *gw, cudaStream_t s);
void launch_check_range(const int32_t *a, int64_t n, int32_t hi, int *flag, cudaStream_t s);

// exec.cu
int enqueue_msf_graph(const DevState &hs, cudaStream_t s, const DevState **host_state);
int enqueue_cc_graph(const DevState &hs, cudaStream_t s, const DevState **host_state);
int run_min_edge_once(const DevState &hs, cudaStream_t s, float *ms);
int run_host_loop(const DevState &hs, cudaStream_t s, const DevState **host_state);
int run_apply_round(const DevState &hs, cudaStream_t s, DevState *out);

}  // namespace msf

// The opaque handle.
struct msf_graph {
  int device;
  int64_t n, m;
  int32_t G;
  int wtype;
  int64_t nnz0, nrows0;
  int32_t build_kernels;  // kernels launched by the build
  int2 *ends;
  int64_t *voff_d, *eoff_d;
  msf::CsrBuf csr0;
  // workspace (allocated on the first compute)
  bool ws_ready;
  msf::CsrBuf w1, w2;
  int32_t *p, *tgt, *changed;
  uint8_t *star;
  int32_t *pjs, *prow;
  int32_t *colr;  // relabelled column words (MSF_OPT_RELABEL), allocated with the workspace
  int32_t *rl_a, *rl_b;
  uint64_t *r, *msf_keys;
  uint32_t *mbits;  // forest-edge bitmap, (m + 31) / 32 + 2 words
  int64_t *rowcnt, *rowflag, *tilecnt, *scan_tmp;
  long long *bins;
  // last run
  msf_stats stats;
};

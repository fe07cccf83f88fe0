// The C ABI (include/msf.h): argument checks, host/device staging, workspace
// and the calls into the device layer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace msf {
const char *last_error_cstr();
}

using namespace msf;

namespace {

constexpr int64_t MAX_N = 2147483647LL;        // vertex ids are int32
constexpr int64_t MAX_M = 4294967294LL;        // edge ids fit in 32 bits below the sentinel

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory (the GPU reads it in place over
// the CPU-GPU link), or NULL.
const void *pinned_host_view(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Device view of a caller buffer: the pointer itself when it is device
// memory (or, with MSF_OPT_HOST_INPUT = 1, page-locked host memory read in
// place), else a pooled device copy (inputs) or scratch (outputs).
struct Staged {
  void *dev = nullptr;
  const void *host_src = nullptr;
  void *host_dst = nullptr;
  size_t bytes = 0;
  bool owned = false;
  ~Staged() {
    if (owned) pool_free(dev);
  }
  int input(const void *p, size_t b, cudaStream_t s) {
    bytes = b;
    if (!p || b == 0 || is_device_ptr(p)) {
      dev = const_cast<void *>(p);
      return MSF_OK;
    }
    if (options().host_input == 1) {
      if (const void *v = pinned_host_view(p)) {
        dev = const_cast<void *>(v);
        return MSF_OK;
      }
    }
    int err = MSF_OK;
    dev = pool_alloc(b, &err);
    if (err) return err;
    owned = true;
    host_src = p;
    MSF_CK(cudaMemcpyAsync(dev, p, b, cudaMemcpyHostToDevice, s));
    return MSF_OK;
  }
  int output(void *p, size_t b) {
    bytes = b;
    if (!p || b == 0 || is_device_ptr(p)) {
      dev = p;
      return MSF_OK;
    }
    int err = MSF_OK;
    dev = pool_alloc(b, &err);
    if (err) return err;
    owned = true;
    host_dst = p;
    return MSF_OK;
  }
  int copy_back(cudaStream_t s) {
    if (host_dst && bytes) MSF_CK(cudaMemcpyAsync(host_dst, dev, bytes, cudaMemcpyDeviceToHost, s));
    return MSF_OK;
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    cudaGetDevice(&now);
    if (prev >= 0 && now != prev) cudaSetDevice(prev);
  }
};

void free_buf(CsrBuf &b) {
  pool_free(b.rows);
  pool_free(b.rp);
  pool_free(b.col);
  pool_free(b.key);
  pool_free(b.tile_row);
  b = CsrBuf{};
}

void free_graph(msf_graph *g) {
  if (!g) return;
  pool_free(g->ends);
  pool_free(g->voff_d);
  pool_free(g->eoff_d);
  free_buf(g->csr0);
  free_buf(g->w1);
  free_buf(g->w2);
  pool_free(g->p);
  pool_free(g->tgt);
  pool_free(g->changed);
  pool_free(g->star);
  pool_free(g->pjs);
  pool_free(g->prow);
  pool_free(g->colr);
  pool_free(g->r);
  pool_free(g->rl_a);
  pool_free(g->rl_b);
  pool_free(g->msf_keys);
  pool_free(g->mbits);
  pool_free(g->rowcnt);
  pool_free(g->rowflag);
  pool_free(g->tilecnt);
  pool_free(g->scan_tmp);
  pool_free(g->bins);
  delete g;
}

int alloc_buf(CsrBuf &b, int64_t cap_slots, int64_t cap_rows) {
  int err = MSF_OK;
  const int64_t padded = (cap_slots + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD + SLOT_PAD;
  b.rows = (int32_t *)pool_alloc((size_t)(cap_rows + 1) * 4, &err);
  if (err) return err;
  b.rp = (int64_t *)pool_alloc((size_t)(cap_rows + 2) * 8, &err);
  if (err) return err;
  b.col = (int32_t *)pool_alloc((size_t)padded * 4, &err);
  if (err) return err;
  b.key = (uint64_t *)pool_alloc((size_t)padded * 8, &err);
  if (err) return err;
  b.tile_row = (int32_t *)pool_alloc((size_t)(padded / TB + 2) * 4, &err);
  if (err) return err;
  b.cap_slots = cap_slots;
  b.cap_rows = cap_rows;
  return MSF_OK;
}

template <class T>
int alloc_n(T **p, int64_t count) {
  int err = MSF_OK;
  *p = (T *)pool_alloc((size_t)(count > 0 ? count : 1) * sizeof(T), &err);
  return err;
}

int ensure_workspace(msf_graph *g) {
  if (g->ws_ready) return MSF_OK;
  const int64_t n = g->n;
  int rc;
  if ((rc = alloc_n(&g->p, n + 1))) return rc;
  if ((rc = alloc_n(&g->tgt, n + 1))) return rc;
  if ((rc = alloc_n(&g->changed, n + 1))) return rc;
  if ((rc = alloc_n(&g->star, n + 1))) return rc;
  if ((rc = alloc_n(&g->prow, g->nrows0 + 1))) return rc;
  if ((rc = alloc_n(&g->colr, (g->nnz0 + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD + SLOT_PAD))) return rc;
  if ((rc = alloc_n(&g->r, n + 1))) return rc;
  if ((rc = alloc_n(&g->rl_a, g->nrows0 + 1))) return rc;
  if ((rc = alloc_n(&g->rl_b, g->nrows0 + 1))) return rc;
  if ((rc = alloc_n(&g->msf_keys, n + 1))) return rc;
  if ((rc = alloc_n(&g->mbits, (g->m + 31) / 32 + 2))) return rc;
  if ((rc = alloc_n(&g->rowcnt, g->nrows0 + 2))) return rc;
  if ((rc = alloc_n(&g->rowflag, g->nrows0 + 2))) return rc;
  if ((rc = alloc_n(&g->tilecnt, g->nnz0 / 128 + 8))) return rc;
  if ((rc = alloc_n(&g->scan_tmp, NB_SCAN + 16))) return rc;
  if ((rc = alloc_n(&g->bins, (int64_t)(g->G > 1 ? g->G : 1 + sum_partials()) * 256))) return rc;
  double capf = options().tau;
  if (capf < 0.5) capf = 0.5;
  if (capf > 1.0) capf = 1.0;
  const int64_t cap = (int64_t)std::ceil(capf * (double)g->nnz0);
  if ((rc = alloc_buf(g->w1, cap, g->nrows0))) return rc;
  if ((rc = alloc_buf(g->w2, cap, g->nrows0))) return rc;
  g->ws_ready = true;
  return MSF_OK;
}

// The pairwise formulation's slot array (nnz0 + padding int32), allocated on
// first use.
int ensure_pairwise(msf_graph *g) {
  if (g->pjs || !options().pairwise) return MSF_OK;
  const int64_t padded = (g->nnz0 + SLOT_PAD - 1) / SLOT_PAD * SLOT_PAD + SLOT_PAD;
  return alloc_n(&g->pjs, padded);
}

DevState make_state(msf_graph *g) {
  DevState hs;
  std::memset(&hs, 0, sizeof(hs));
  const Options &o = options();
  hs.n = g->n;
  hs.m = g->m;
  hs.G = g->G;
  hs.wtype = g->wtype;
  hs.voff = g->voff_d;
  hs.eoff = g->eoff_d;
  hs.ends = g->ends;
  hs.buf[0] = g->csr0;
  hs.buf[1] = g->w1;
  hs.buf[2] = g->w2;
  hs.cur = 0;
  hs.nrows = g->nrows0;
  hs.nnz = g->nnz0;
  hs.p = g->p;
  hs.tgt = g->tgt;
  hs.r = g->r;
  hs.rl = g->csr0.rows;
  hs.rl_n = (unsigned long long)g->nrows0;
  hs.nrows0 = g->nrows0;
  hs.rl_buf[0] = g->rl_a;
  hs.rl_buf[1] = g->rl_b;
  hs.rl_next = g->rl_a;
  hs.rl_all = o.shortcut_mode == MSF_SHORTCUT_ORIGINAL ? 1 : 0;
  hs.changed = g->changed;
  hs.msf_keys = g->msf_keys;
  hs.rowcnt = g->rowcnt;
  hs.rowflag = g->rowflag;
  hs.tilecnt = g->tilecnt;
  hs.scan_tmp = g->scan_tmp;
  hs.bins = g->bins;
  hs.round_limit = o.round_limit;
  hs.jump_limit = o.jump_limit;
  hs.tau = (float)o.tau;
  hs.spl = o.spl;
  hs.first_round_identity = 1;
  hs.shortcut_mode = o.shortcut_mode;
  hs.os_threshold = o.os_threshold;
  hs.star = (o.shortcut_mode == MSF_SHORTCUT_ORIGINAL) ? g->star : nullptr;
  hs.pjs = g->pjs;
  hs.prow = g->prow;
  // the relabelled columns serve the register sweeps of the multilinear kernel
  hs.colr = (o.relabel && !o.pairwise && o.sweep == 0 && o.shortcut_mode != MSF_SHORTCUT_ORIGINAL) ? g->colr
                                                                                                    : nullptr;
  hs.early_stop = o.early_stop;
  return hs;
}

int check_weights_type(int wtype) {
  if (wtype != MSF_F32 && wtype != MSF_U32) return fail(MSF_ERR_INVALID_ARG, "wtype must be MSF_F32 or MSF_U32");
  return MSF_OK;
}

int graph_compute(msf_graph *g, uint8_t *edge_mask, int32_t *labels, double *totals, int64_t ntot,
                  cudaStream_t s) {
  int rc = ensure_workspace(g);
  if (rc) return rc;
  if ((rc = ensure_pairwise(g))) return rc;
  Staged sm, sl, st;
  if ((rc = sm.output(edge_mask, (size_t)g->m))) return rc;
  if ((rc = sl.output(labels, (size_t)g->n * 4))) return rc;
  if ((rc = st.output(totals, (size_t)ntot * 8))) return rc;
  DevState hs = make_state(g);
  hs.mask = (uint8_t *)sm.dev;
  hs.mbits = g->mbits;
  hs.labels = (int32_t *)sl.dev;
  hs.totals = (double *)st.dev;
  const DevState *back = nullptr;
  if (options().exec_mode == 1) {
    if ((rc = run_host_loop(hs, s, &back))) return rc;
  } else {
    if ((rc = enqueue_msf_graph(hs, s, &back))) return rc;
  }
  if ((rc = sm.copy_back(s))) return rc;
  if ((rc = sl.copy_back(s))) return rc;
  if ((rc = st.copy_back(s))) return rc;
  MSF_CK(cudaStreamSynchronize(s));
  g->stats.n = g->n;
  g->stats.m = g->m;
  g->stats.nnz = g->nnz0;
  g->stats.rows = g->nrows0;
  g->stats.rounds = back->round;
  g->stats.compactions = back->compactions;
  g->stats.forest_edges = (int64_t)back->n_msf;
  g->stats.jump_steps = back->jumps_total;
  {
    // kernels of the round loop: per round the sweep with its row parents,
    // hooking, tie breaking and the schedule's shortcut and control steps,
    // two per shortcut pass, 16 per compaction; then labels, mask and sums
    const Options &o = options();
    int per_round = 0;
    switch (o.shortcut_mode) {
      case MSF_SHORTCUT_ORIGINAL: per_round = 12; break;
      case MSF_SHORTCUT_FULL: per_round = 7; break;
      case MSF_SHORTCUT_OPTIMIZED: per_round = 9; break;
      default: per_round = 8; break;
    }
    if (o.pairwise) per_round += 1;
    else if (o.sweep == 0) per_round += 1;  // the register sweep's relabelling instantiation
    g->stats.kernels = g->build_kernels + 1 /* state upload */ + 1 /* init */ + per_round * back->round +
                       2 * back->jumps_total + 16 * back->compactions +
                       7 /* labels (3), mask bits and expansion, sum, finalize */;
  }
  switch (back->status) {
    case MSF_OK: return MSF_OK;
    case MSF_ERR_ROUND_LIMIT: return fail(MSF_ERR_ROUND_LIMIT, "round limit reached before the forest converged");
    case MSF_ERR_SHORTCUT_LIMIT: return fail(MSF_ERR_SHORTCUT_LIMIT, "pointer jumping did not settle within the limit");
    default: return fail(back->status, "device consistency check failed");
  }
}

int build_graph_common(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *row_ptr,
                       const void *w, int wtype, int32_t G, const int64_t *voff_h, const int64_t *eoff_h,
                       cudaStream_t s, msf_graph **out) {
  int rc;
  msf_graph *g = new msf_graph();
  std::memset(g, 0, sizeof(*g));
  cudaGetDevice(&g->device);
  g->n = n;
  g->m = m;
  g->G = G;
  g->wtype = wtype;
  Staged ss, sd, sw, sr;
  if ((rc = sd.input(dst, (size_t)m * 4, s)) || (rc = sw.input(w, (size_t)m * 4, s)) ||
      (!row_ptr && (rc = ss.input(src, (size_t)m * 4, s))) ||
      (row_ptr && (rc = sr.input(row_ptr, (size_t)(n + 1) * 8, s)))) {
    cudaStreamSynchronize(s);  // copies already queued finish before their buffers return to the pool
    free_graph(g);
    return rc;
  }
  if (row_ptr) {
    int64_t ends2[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&ends2[0], sr.dev, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends2[1], (const int64_t *)sr.dev + n, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      free_graph(g);
      return cuda_fail(e, "reading row_ptr");
    }
    if (ends2[0] != 0 || ends2[1] != m) {
      free_graph(g);
      return fail(MSF_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] must equal m");
    }
  }
  if (G > 1) {
    // the offsets, each followed by its block table (internal.cuh)
    int err = MSF_OK;
    g->voff_d = (int64_t *)pool_alloc((size_t)(G + 1) * 8 + (size_t)(off_table_len(n) + 1) * 4, &err);
    if (!err) g->eoff_d = (int64_t *)pool_alloc((size_t)(G + 1) * 8 + (size_t)(off_table_len(m) + 1) * 4, &err);
    if (err) {
      free_graph(g);
      return err;
    }
    cudaError_t e = cudaMemcpyAsync(g->voff_d, voff_h, (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->eoff_d, eoff_h, (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      launch_off_table(g->voff_d, G, n, s);
      launch_off_table(g->eoff_d, G, m, s);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      free_graph(g);
      return cuda_fail(e, "copying offsets");
    }
  }
  rc = build_csr_device(n, m, (const int32_t *)ss.dev, (const int32_t *)sd.dev, (const int64_t *)sr.dev, sw.dev,
                        wtype, G, g->eoff_d, g->voff_d, s, g);
  if (rc) {
    free_graph(g);
    return rc;
  }
  *out = g;
  return MSF_OK;
}

}  // namespace

extern "C" {

const char *msf_last_error(void) { return last_error_cstr(); }

int msf_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const int64_t *row_ptr,
                  const void *w, int wtype, uint32_t flags, void *stream, msf_graph **out) {
  set_error("");
  if (!out) return fail(MSF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 0 || m < 0) return fail(MSF_ERR_INVALID_ARG, "n and m must be non-negative");
  if (n > MAX_N || m > MAX_M) return fail(MSF_ERR_TOO_LARGE, "n must be < 2^31 and m < 2^32 - 1");
  if (flags != 0) return fail(MSF_ERR_INVALID_ARG, "flags must be 0");
  if (int rc = check_weights_type(wtype)) return rc;
  if (m > 0 && (!dst || !w || (!row_ptr && !src))) return fail(MSF_ERR_INVALID_ARG, "NULL edge array");
  if (m > 0 && n == 0) return fail(MSF_ERR_INVALID_ARG, "edges given for an empty vertex set");
  return build_graph_common(n, m, src, dst, row_ptr, w, wtype, 1, nullptr, nullptr, (cudaStream_t)stream, out);
}

int msf_compute(msf_graph *g, uint8_t *edge_mask, int32_t *labels, double *total, void *stream) {
  set_error("");
  if (!g) return fail(MSF_ERR_INVALID_ARG, "graph is NULL");
  DeviceGuard dg(g->device);
  return graph_compute(g, edge_mask, labels, total, 1, (cudaStream_t)stream);
}

int msf_compute_batched(int32_t G, const int64_t *voff, const int64_t *eoff, const int32_t *src,
                        const int32_t *dst, const void *w, int wtype, uint8_t *edge_mask, int32_t *labels,
                        double *totals, void *stream) {
  set_error("");
  if (G < 0) return fail(MSF_ERR_INVALID_ARG, "G must be non-negative");
  if (G == 0) return MSF_OK;
  if (!voff || !eoff) return fail(MSF_ERR_INVALID_ARG, "voff and eoff are required");
  if (is_device_ptr(voff) || is_device_ptr(eoff)) return fail(MSF_ERR_INVALID_ARG, "voff and eoff must be host arrays");
  if (int rc = check_weights_type(wtype)) return rc;
  if (voff[0] != 0 || eoff[0] != 0) return fail(MSF_ERR_INVALID_ARG, "voff[0] and eoff[0] must be 0");
  for (int32_t g = 0; g < G; ++g)
    if (voff[g + 1] < voff[g] || eoff[g + 1] < eoff[g]) return fail(MSF_ERR_INVALID_ARG, "offsets must be non-decreasing");
  const int64_t n = voff[G], m = eoff[G];
  if (n > MAX_N || m > MAX_M) return fail(MSF_ERR_TOO_LARGE, "total n must be < 2^31 and total m < 2^32 - 1");
  if (m > 0 && (!src || !dst || !w)) return fail(MSF_ERR_INVALID_ARG, "NULL edge array");
  cudaStream_t s = (cudaStream_t)stream;
  msf_graph *g = nullptr;
  int rc = build_graph_common(n, m, src, dst, nullptr, w, wtype, G, voff, eoff, s, &g);
  if (rc) return rc;
  rc = graph_compute(g, edge_mask, labels, totals, G, s);
  free_graph(g);
  return rc;
}

void msf_free(msf_graph *g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  free_graph(g);
}

int msf_min_edge(msf_graph *g, const int32_t *parent, uint64_t *r, void *stream) {
  set_error("");
  if (!g || !parent || !r) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  Staged sp, sr;
  if ((rc = sp.input(parent, (size_t)g->n * 4, s))) return rc;
  if ((rc = sr.output(r, (size_t)g->n * 8))) return rc;
  int err = MSF_OK;
  int *flag = (int *)pool_alloc(16, &err);
  if (err) return err;
  int hflag = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, 4, s);
  if (e == cudaSuccess && g->n > 0) {
    launch_check_range((const int32_t *)sp.dev, g->n, (int32_t)g->n, flag, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  pool_free(flag);
  if (e != cudaSuccess) return cuda_fail(e, "checking parent");
  if (hflag) return fail(MSF_ERR_INVALID_ARG, "parent value outside [0, n)");
  if (g->n > 0) MSF_CK(cudaMemsetAsync(sr.dev, 0xff, (size_t)g->n * 8, s));
  DevState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.n = g->n;
  hs.m = g->m;
  hs.G = g->G;
  hs.wtype = g->wtype;
  hs.buf[0] = g->csr0;
  hs.cur = 0;
  hs.nrows = g->nrows0;
  hs.nnz = g->nnz0;
  hs.p = (int32_t *)sp.dev;
  hs.r = (uint64_t *)sr.dev;
  hs.first_round_identity = 0;
  if ((rc = ensure_pairwise(g))) return rc;
  if ((rc = ensure_workspace(g))) return rc;
  hs.pjs = g->pjs;
  hs.prow = g->prow;
  float ms = 0.f;
  if ((rc = run_min_edge_once(hs, s, &ms))) return rc;
  g->stats.min_edge_ms = ms;
  if ((rc = sr.copy_back(s))) return rc;
  MSF_CK(cudaStreamSynchronize(s));
  return MSF_OK;
}

int msf_min_edge_part(msf_graph *g, const int32_t *parent, int32_t part, int32_t nparts, uint64_t *r,
                      void *stream) {
  set_error("");
  if (!g || !parent || !r) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  if (nparts < 1 || part < 0 || part >= nparts) return fail(MSF_ERR_INVALID_ARG, "need 0 <= part < nparts");
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  Staged sp, sr;
  if ((rc = sp.input(parent, (size_t)g->n * 4, s))) return rc;
  if ((rc = sr.output(r, (size_t)g->n * 8))) return rc;
  int err = MSF_OK;
  int *flag = (int *)pool_alloc(16, &err);
  if (err) return err;
  int hflag = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, 4, s);
  if (e == cudaSuccess && g->n > 0) {
    launch_check_range((const int32_t *)sp.dev, g->n, (int32_t)g->n, flag, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  pool_free(flag);
  if (e != cudaSuccess) return cuda_fail(e, "checking parent");
  if (hflag) return fail(MSF_ERR_INVALID_ARG, "parent value outside [0, n)");
  if (g->n > 0) MSF_CK(cudaMemsetAsync(sr.dev, 0xff, (size_t)g->n * 8, s));
  // the part's slots [s0, s1): cuts at multiples of SLOT_PAD, so that every
  // tile of the sweep (at most SLOT_PAD slots) lies inside one part
  const int64_t nnz = g->nnz0;
  auto cut = [&](int64_t k) -> int64_t {
    if (k >= nparts) return nnz;
    const int64_t c = (int64_t)((__int128)k * nnz / nparts);
    return c / SLOT_PAD * SLOT_PAD;
  };
  const int64_t s0 = cut(part), s1 = cut((int64_t)part + 1);
  if (s1 > s0) {
    if ((rc = ensure_workspace(g))) return rc;
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.n = g->n;
    hs.m = g->m;
    hs.G = g->G;
    hs.wtype = g->wtype;
    // a view of the original CSR that starts at slot s0 (tile_row is indexed
    // by slot / TB and s0 is a multiple of TB); rows, rp and the row parents
    // stay global
    hs.buf[0] = g->csr0;
    hs.buf[0].col += s0;
    hs.buf[0].key += s0;
    hs.buf[0].tile_row += s0 / TB;
    hs.cur = 0;
    hs.nrows = g->nrows0;
    hs.nnz = s1 - s0;
    hs.p = (int32_t *)sp.dev;
    hs.r = (uint64_t *)sr.dev;
    hs.first_round_identity = 0;
    hs.prow = g->prow;
    if (options().pairwise) {
      if ((rc = ensure_pairwise(g))) return rc;
      hs.pjs = g->pjs;
    }
    float ms = 0.f;
    if ((rc = run_min_edge_once(hs, s, &ms))) return rc;
    g->stats.min_edge_ms = ms;
  }
  if ((rc = sr.copy_back(s))) return rc;
  MSF_CK(cudaStreamSynchronize(s));
  return MSF_OK;
}

int msf_apply_round(msf_graph *g, uint64_t *r, int32_t *parent, uint8_t *edge_mask, int32_t *labels,
                    int64_t *hooks, void *stream) {
  set_error("");
  if (!g || !r || !parent || !edge_mask || !hooks) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(g->device);
  if (g->n > 0 && (!is_device_ptr(r) || !is_device_ptr(parent) || (labels && !is_device_ptr(labels))))
    return fail(MSF_ERR_INVALID_ARG, "r, parent and labels must be device memory");
  if (g->m > 0 && !is_device_ptr(edge_mask)) return fail(MSF_ERR_INVALID_ARG, "edge_mask must be device memory");
  *hooks = 0;
  if (g->n == 0) return MSF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_workspace(g);
  if (rc) return rc;
  DevState hs = make_state(g);
  // every vertex is visited (no root list is kept between calls)
  hs.rl_all = 1;
  hs.rl = nullptr;
  hs.p = parent;
  hs.r = r;
  hs.mask = edge_mask;
  hs.labels = labels;
  hs.totals = nullptr;
  hs.star = nullptr;
  hs.first_round_identity = 0;
  hs.shortcut_mode = MSF_SHORTCUT_CSP;
  hs.early_stop = 0;
  hs.tau = 0.f;
  hs.colr = nullptr;
  DevState back;
  if ((rc = run_apply_round(hs, s, &back))) return rc;
  *hooks = (int64_t)back.n_msf;
  if (back.status == MSF_ERR_SHORTCUT_LIMIT) return fail(MSF_ERR_SHORTCUT_LIMIT, "shortcutting did not settle");
  if (back.status) return fail(back.status, "a key of r does not leave its star");
  return MSF_OK;
}

int msf_connected_components(msf_graph *g, int32_t *labels, void *stream) {
  set_error("");
  if (!g || !labels) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_workspace(g);
  if (rc) return rc;
  Staged sl;
  if ((rc = sl.output(labels, (size_t)g->n * 4))) return rc;
  DevState hs = make_state(g);
  hs.labels = (int32_t *)sl.dev;
  hs.mask = nullptr;
  hs.totals = nullptr;
  hs.star = g->star;
  hs.tau = 0.f;
  hs.early_stop = 0;
  hs.colr = nullptr;
  const DevState *back = nullptr;
  if ((rc = enqueue_cc_graph(hs, s, &back))) return rc;
  if ((rc = sl.copy_back(s))) return rc;
  MSF_CK(cudaStreamSynchronize(s));
  g->stats.cc_rounds = back->round;
  if (back->status == MSF_ERR_ROUND_LIMIT) return fail(MSF_ERR_ROUND_LIMIT, "round limit reached");
  if (back->status == MSF_ERR_SHORTCUT_LIMIT) return fail(MSF_ERR_SHORTCUT_LIMIT, "shortcutting did not settle");
  if (back->status) return fail(back->status, "device consistency check failed");
  return MSF_OK;
}

int msf_weight_backward(int64_t m, int32_t G, const int64_t *eoff, const uint8_t *edge_mask,
                        const double *grad_total, float *grad_w, void *stream) {
  set_error("");
  if (m < 0 || G < 1) return fail(MSF_ERR_INVALID_ARG, "m must be >= 0 and G >= 1");
  if (m == 0) return MSF_OK;
  if (!edge_mask || !grad_total || !grad_w) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  if (G > 1 && !eoff) return fail(MSF_ERR_INVALID_ARG, "eoff is required when G > 1");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  Staged se, sm, sg, sw;
  if (G > 1 && (rc = se.input(eoff, (size_t)(G + 1) * 8, s))) return rc;
  if ((rc = sm.input(edge_mask, (size_t)m, s))) return rc;
  if ((rc = sg.input(grad_total, (size_t)G * 8, s))) return rc;
  if ((rc = sw.output(grad_w, (size_t)m * 4))) return rc;
  launch_backward(m, G, (const int64_t *)se.dev, (const uint8_t *)sm.dev, (const double *)sg.dev,
                  (float *)sw.dev, s);
  MSF_CK(cudaGetLastError());
  if ((rc = sw.copy_back(s))) return rc;
  if (se.owned || sm.owned || sg.owned || sw.owned) MSF_CK(cudaStreamSynchronize(s));
  return MSF_OK;
}

int msf_get_stats(const msf_graph *g, msf_stats *out) {
  set_error("");
  if (!g || !out) return fail(MSF_ERR_INVALID_ARG, "NULL argument");
  *out = g->stats;
  out->n = g->n;
  out->m = g->m;
  out->nnz = g->nnz0;
  out->rows = g->nrows0;
  return MSF_OK;
}

int msf_set_option(int option, double value) {
  Options &o = options();
  switch (option) {
    case MSF_OPT_COMPACT_TAU:
      if (!(value >= 0.0 && value < 1.0)) return fail(MSF_ERR_INVALID_ARG, "tau must be in [0, 1)");
      o.tau = value;
      return MSF_OK;
    case MSF_OPT_ROUND_LIMIT:
      if (!(value >= 1 && value <= 1024)) return fail(MSF_ERR_INVALID_ARG, "round limit must be in [1, 1024]");
      o.round_limit = (int)value;
      return MSF_OK;
    case MSF_OPT_JUMP_LIMIT:
      if (!(value >= 1 && value <= 1024)) return fail(MSF_ERR_INVALID_ARG, "jump limit must be in [1, 1024]");
      o.jump_limit = (int)value;
      return MSF_OK;
    case MSF_OPT_SLOTS_PER_LANE:
      if (value != 4 && value != 8 && value != 16) return fail(MSF_ERR_INVALID_ARG, "slots per lane must be 4, 8 or 16");
      o.spl = (int)value;
      return MSF_OK;
    case MSF_OPT_BLOCKS_PER_SM:
      if (!(value >= 1 && value <= 8)) return fail(MSF_ERR_INVALID_ARG, "blocks per SM must be in [1, 8]");
      o.blocks_per_sm = (int)value;
      return MSF_OK;
    case MSF_OPT_PREFETCH:
      if (value != 0 && value != 1) return fail(MSF_ERR_INVALID_ARG, "prefetch must be 0 or 1");
      o.prefetch = (int)value;
      return MSF_OK;
    case MSF_OPT_EXEC_MODE:
      if (value != 0 && value != 1) return fail(MSF_ERR_INVALID_ARG, "exec mode must be 0 (graph) or 1 (host loop)");
      o.exec_mode = (int)value;
      return MSF_OK;
    case MSF_OPT_SHORTCUT:
      if (!(value == 0 || value == 1 || value == 2 || value == 3))
        return fail(MSF_ERR_INVALID_ARG, "shortcut schedule must be one of MSF_SHORTCUT_*");
      o.shortcut_mode = (int)value;
      return MSF_OK;
    case MSF_OPT_EARLY_STOP:
      if (value != 0 && value != 1) return fail(MSF_ERR_INVALID_ARG, "early stop must be 0 or 1");
      o.early_stop = (int)value;
      return MSF_OK;
    case MSF_OPT_SWEEP:
      if (value != 0 && value != 1 && value != 2) return fail(MSF_ERR_INVALID_ARG, "sweep form must be 0, 1 or 2");
      o.sweep = (int)value;
      return MSF_OK;
    case MSF_OPT_HOST_INPUT:
      if (value != 0 && value != 1) return fail(MSF_ERR_INVALID_ARG, "host input mode must be 0 or 1");
      o.host_input = (int)value;
      return MSF_OK;
    case MSF_OPT_RELABEL:
      if (value != 0 && value != 1) return fail(MSF_ERR_INVALID_ARG, "relabel must be 0 or 1");
      o.relabel = (int)value;
      return MSF_OK;
    case MSF_OPT_BUILD:
      if (!(value == 0 || value == 1 || value == 2 || value == 3))
        return fail(MSF_ERR_INVALID_ARG, "build mode must be 0, 1, 2 or 3");
      o.build_mode = (int)value;
      return MSF_OK;
    case MSF_OPT_KERNEL:
      if (value != 0 && value != 1) return fail(MSF_ERR_INVALID_ARG, "kernel must be 0 (multilinear) or 1 (pairwise)");
      o.pairwise = (int)value;
      return MSF_OK;
    case MSF_OPT_OS_THRESHOLD:
      if (!(value >= 0 && value <= 9.2e18)) return fail(MSF_ERR_INVALID_ARG, "threshold must be >= 0");
      o.os_threshold = (int64_t)value;
      return MSF_OK;
    default:
      return fail(MSF_ERR_INVALID_ARG, "unknown option");
  }
}

double msf_get_option(int option) {
  const Options &o = options();
  switch (option) {
    case MSF_OPT_COMPACT_TAU: return o.tau;
    case MSF_OPT_ROUND_LIMIT: return o.round_limit;
    case MSF_OPT_JUMP_LIMIT: return o.jump_limit;
    case MSF_OPT_SLOTS_PER_LANE: return o.spl;
    case MSF_OPT_BLOCKS_PER_SM: return o.blocks_per_sm;
    case MSF_OPT_PREFETCH: return o.prefetch;
    case MSF_OPT_EXEC_MODE: return o.exec_mode;
    case MSF_OPT_SHORTCUT: return o.shortcut_mode;
    case MSF_OPT_OS_THRESHOLD: return (double)o.os_threshold;
    case MSF_OPT_KERNEL: return o.pairwise;
    case MSF_OPT_BUILD: return o.build_mode;
    case MSF_OPT_EARLY_STOP: return o.early_stop;
    case MSF_OPT_SWEEP: return o.sweep;
    case MSF_OPT_HOST_INPUT: return o.host_input;
    case MSF_OPT_RELABEL: return o.relabel;
    default: return -1.0;
  }
}

}  // extern "C"
